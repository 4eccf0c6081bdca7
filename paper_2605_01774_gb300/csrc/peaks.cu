// CUDA-core fused multiply-add throughput of the current device, measured: the arithmetic
// roofline against which the FP64 step (bound by FP64 FMA issue, not HBM) is placed.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/elbm.h"

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

}  // namespace

extern "C" elbm_status elbm_fma_peak(int32_t precision, double* flops_per_s) {
  if (!flops_per_s) return ELBM_ERR_ARG;
  if (precision == ELBM_F64) return run<double>(flops_per_s);
  if (precision == ELBM_F32) return run<float>(flops_per_s);
  return ELBM_ERR_ARG;
}
