// CUDA-core fused multiply-add throughput of the current device, measured: the arithmetic
// roofline against which the FP64 step (bound by FP64 FMA issue, not HBM) is placed.  And the
// rate at which warps issue bulk asynchronous global -> shared copies, which sets how the
// staged-row step spreads a row's copies over its warps.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/elbm.h"
#include "bulk.cuh"

namespace {

constexpr int CHAINS = 8;       // independent FMA chains per thread (hides the FMA latency)
constexpr int ITERS = 4096;     // iterations per chain
constexpr int THREADS = 256;

__device__ double g_sink;       // keeps the chains live; written only if the result is NaN

template <typename T>
__global__ void __launch_bounds__(THREADS) k_fma_peak(T b, T c) {
  T a[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) a[j] = T(threadIdx.x + j);
#pragma unroll 4
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) a[j] = fma(a[j], b, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) s += a[j];
  if (s != s) g_sink = double(s);
}

template <typename T>
elbm_status run(double* flops_per_s) {
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, THREADS, 0) != cudaSuccess)
    return ELBM_ERR_CUDA;
  const int grid = nsm * std::max(per_sm, 1) * 4;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return ELBM_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // b slightly below 1 and c small keep the chains finite and non-denormal
  const T b = T(0.999999), c = T(1e-3);
  double best = 0.0;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 6 && err == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_peak<T><<<grid, THREADS, 0, s>>>(b, c);
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0 && ms > 0.f)   // first launch is a warm-up
      best = std::max(best, 2.0 * CHAINS * ITERS * double(grid) * THREADS / (ms * 1e-3));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (err != cudaSuccess) return ELBM_ERR_CUDA;
  *flops_per_s = best;
  return ELBM_OK;
}

// Bulk-copy throughput: persistent blocks, each of whose warp 0 issues the copies of one stage
// (copy_bytes each, about 24 KiB per stage, two stages) and refills a stage once the block has
// read it; every wait is bounded.  One launch reads `iters` stages per block from a source larger
// than L2.
constexpr int BC_THREADS = 256;
constexpr int BC_STAGE = 24 * 1024;

__global__ void __launch_bounds__(BC_THREADS) k_bulk_rate(const unsigned char* __restrict__ src, size_t nchunks,
                                                          int copy_bytes, int per_stage, int iters,
                                                          unsigned* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bar[2];
  if (threadIdx.x == 0) {
    elbm::mbar_init(&bar[0], 1);
    elbm::mbar_init(&bar[1], 1);
    elbm::mbar_fence_init();
  }
  __syncthreads();
  const size_t stage = (size_t)copy_bytes * per_stage;
  size_t chunk = blockIdx.x;
  auto issue = [&](int it) {
    const int s = it & 1;
    const unsigned char* g = src + (chunk % nchunks) * stage;
    if (threadIdx.x == 0) elbm::mbar_arrive_expect_tx(&bar[s], (uint32_t)stage);
    __syncwarp();
    for (int c = threadIdx.x; c < per_stage; c += 32)
      elbm::bulk_copy_g2s(sm + s * stage + (size_t)c * copy_bytes, g + (size_t)c * copy_bytes, copy_bytes, &bar[s]);
    chunk += gridDim.x;
  };
  if (threadIdx.x < 32)
    for (int it = 0; it < 2 && it < iters; ++it) issue(it);
  float acc = 0.f;
  for (int it = 0; it < iters; ++it) {
    const int s = it & 1;
    const bool ok = elbm::mbar_wait_bounded(&bar[s], (it >> 1) & 1, 2000000000ll);
    acc += reinterpret_cast<const float*>(sm + s * stage)[threadIdx.x % (stage / 4)];
    // the barrier orders the reads of the stage before its refill and makes the outcome of the
    // waits block-uniform
    if (__syncthreads_or(ok ? 0 : 1)) {
      if (threadIdx.x == 0) {
        // leave no copy in flight: the stages of iterations it and it + 1
        atomicAdd(err, 1u);
        elbm::mbar_wait_bounded(&bar[s], (it >> 1) & 1, 2000000000ll);
        if (it + 1 < iters) elbm::mbar_wait_bounded(&bar[s ^ 1], ((it + 1) >> 1) & 1, 2000000000ll);
      }
      break;
    }
    if (threadIdx.x < 32 && it + 2 < iters) issue(it + 2);
  }
  if (acc != acc) atomicAdd(err, 2u);
}

}  // namespace

extern "C" elbm_status elbm_bulk_copy_rate(int32_t copy_bytes, int32_t blocks_per_sm, double* bytes_per_s,
                                           double* copies_per_s) {
  if (!bytes_per_s || !copies_per_s || copy_bytes < 16 || copy_bytes > BC_STAGE || copy_bytes % 16 != 0 ||
      blocks_per_sm < 1 || blocks_per_sm > 4)
    return ELBM_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ELBM_ERR_CUDA;
  const int per_stage = BC_STAGE / copy_bytes;
  const size_t stage = (size_t)copy_bytes * per_stage, dyn = 2 * stage;
  const size_t src_bytes = 1ull << 30;          // 1 GiB source: larger than L2
  const size_t nchunks = src_bytes / stage;
  const int grid = nsm * blocks_per_sm;
  const int iters = (int)(nchunks / grid);
  unsigned char* src = nullptr;
  unsigned* err = nullptr;
  if (cudaMalloc(&src, src_bytes) != cudaSuccess) return ELBM_ERR_OOM;
  if (cudaMalloc(&err, sizeof(unsigned)) != cudaSuccess) {
    cudaFree(src);
    return ELBM_ERR_OOM;
  }
  cudaStream_t s;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(src, 1, src_bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bulk_rate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    k_bulk_rate<<<grid, BC_THREADS, dyn, s>>>(src, nchunks, copy_bytes, per_stage, iters, err);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms > 0.f)   // first launch is a warm-up
      best = std::max(best, (double)iters * grid * stage / (ms * 1e-3));
  }
  unsigned h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaFree(src);
  cudaFree(err);
  if (e != cudaSuccess) return ELBM_ERR_CUDA;
  if (h != 0) return ELBM_ERR_TIMEOUT;
  *bytes_per_s = best;
  *copies_per_s = best / copy_bytes;
  return ELBM_OK;
}

extern "C" elbm_status elbm_fma_peak(int32_t precision, double* flops_per_s) {
  if (!flops_per_s) return ELBM_ERR_ARG;
  if (precision == ELBM_F64) return run<double>(flops_per_s);
  if (precision == ELBM_F32) return run<float>(flops_per_s);
  return ELBM_ERR_ARG;
}
