// Conservation diagnostics of a caller-held population state without any device
// allocation: a grid-stride variant of the reduction in aux.cu whose partial sums
// live in a file-scope device array instead of a buffer from cudaMalloc.
//
// Who needs it: code that must not allocate device memory at the moment it wants
// the diagnostics -- a process whose device memory is already fully reserved by
// another allocator (a framework's caching allocator or a memory pool that owns the
// GPU), or a monitoring hook inside a time-stepping loop where an allocation that
// blocks or fails is not acceptable (e.g. reporting after an out-of-memory error).
#include <cmath>
#include <mutex>

#include "../../include/elbm.h"
#include "internal.h"
#include "pull.cuh"

using namespace elbm;

namespace {

constexpr int kMaxPartials = 4096;  // blocks of the partial-sum kernel (grid-stride over nodes)
constexpr int kMaxDevices = 64;

// 4 doubles per block (mass, entropy, min g, non-finite count) + 4 for the final result:
// 131 104 bytes on every GPU that loads the library, held until the process exits.
__device__ __align__(256) double g_scratch[4 * kMaxPartials + 4];

std::mutex g_mu;
// Device address of g_scratch per device, and the id of the context it was looked up in: a
// module's __device__ arrays are placed anew when a device's context is destroyed and
// re-created (cudaDeviceReset), so the address is looked up again when the id changes.
double* g_scratch_dev[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

template <typename Elem>
__global__ void __launch_bounds__(256)
k_partials_strided(Field<Elem> f, Grid G, const float* __restrict__ src, double* __restrict__ part,
                   const PopConsts<typename Storage<Elem>::real> k) {
  using R = typename Storage<Elem>::real;
  double m = 0.0, h = 0.0, gmin = 1.7976931348623157e308, bad = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < G.N; n += stride) {
    const int x = (int)(n % G.nx);
    const int y = (int)((n / G.nx) % G.ny);
    const int z = (int)(n / ((size_t)G.nx * G.ny));
    R g[Q];
    pull_node<Elem, R>(g, f, G, x, y, z, k);
    const double r = src != nullptr ? 0.5 * (double)src[n] : 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double v = (double)g[i] + r * (double)k.E[i];
      if (!isfinite(v)) {
        bad += 1.0;
        continue;
      }
      m += v;
      if (v > 0.0) h += v * log(v / w_of(i));
      gmin = fmin(gmin, v);
    }
  }
  __shared__ double sm[4][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_xor_sync(0xffffffffu, m, o);
    h += __shfl_xor_sync(0xffffffffu, h, o);
    gmin = fmin(gmin, __shfl_xor_sync(0xffffffffu, gmin, o));
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (lane == 0) {
    sm[0][wid] = m;
    sm[1][wid] = h;
    sm[2][wid] = gmin;
    sm[3][wid] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 1.7976931348623157e308, d = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      a += sm[0][w];
      b += sm[1][w];
      c = fmin(c, sm[2][w]);
      d += sm[3][w];
    }
    part[4 * blockIdx.x + 0] = a;
    part[4 * blockIdx.x + 1] = b;
    part[4 * blockIdx.x + 2] = c;
    part[4 * blockIdx.x + 3] = d;
  }
}

__global__ void __launch_bounds__(256) k_final_strided(const double* __restrict__ part, int nblk,
                                                       double* __restrict__ out4) {
  __shared__ double sm[4][256];
  double a = 0, b = 0, c = 1.7976931348623157e308, d = 0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    a += part[4 * i];
    b += part[4 * i + 1];
    c = fmin(c, part[4 * i + 2]);
    d += part[4 * i + 3];
  }
  sm[0][threadIdx.x] = a;
  sm[1][threadIdx.x] = b;
  sm[2][threadIdx.x] = c;
  sm[3][threadIdx.x] = d;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + s];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + s];
      sm[2][threadIdx.x] = fmin(sm[2][threadIdx.x], sm[2][threadIdx.x + s]);
      sm[3][threadIdx.x] += sm[3][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out4[0] = sm[0][0];
    out4[1] = sm[1][0];
    out4[2] = sm[2][0];
    out4[3] = sm[3][0];
  }
}

// Unique id of the current context (driver entry points fetched through the runtime, so the
// library needs no link against the driver library); 0 if it cannot be had.
unsigned long long current_context_id() {
  typedef int (*get_current_t)(void**);
  typedef int (*get_id_t)(void*, unsigned long long*);
  static get_current_t get_current = nullptr;
  static get_id_t get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<get_current_t>(f1);
      get_id = reinterpret_cast<get_id_t>(f2);
    }
    cudaGetLastError();
    looked_up = true;
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == 0 && ctx != nullptr && get_id(ctx, &id) == 0) return id;
  return 0;
}

// Device address of g_scratch on the current device: looked up (cudaGetSymbolAddress, with
// the device current) on the first call in each context of that device, then cached.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long ctx = current_context_id();
  if (g_scratch_dev[dev] == nullptr || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
    // the symbol lookup made the runtime create the context if there was none yet
    g_scratch_ctx[dev] = ctx != 0 ? ctx : current_context_id();
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

template <typename R>
PopConsts<R> pull_consts(const double u[3], const elbm_bc* bc) {
  PopConsts<R> k{};
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    const double cu = cx_of(i) * u[0] + cy_of(i) * u[1] + cz_of(i) * u[2];
    k.E[i] = (R)(w_of(i) * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
  }
  k.phi_lo = (R)(bc ? bc->phi_lo : 0.0);
  k.phi_hi = (R)(bc ? bc->phi_hi : 0.0);
  return k;
}

template <typename Elem>
cudaError_t launch(const void* pops, const float* scale, const Grid& G, const float* src, const double u[3],
                   const elbm_bc* bc, double* scratch, double* out4, cudaStream_t s) {
  using R = typename Storage<Elem>::real;
  const size_t want = (G.N + 255) / 256;
  const int nblk = (int)(want < (size_t)kMaxPartials ? want : (size_t)kMaxPartials);
  Field<Elem> f{static_cast<const Elem*>(pops), scale};
  k_partials_strided<Elem><<<nblk, 256, 0, s>>>(f, G, src, scratch, pull_consts<R>(u, bc));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_final_strided<<<1, 256, 0, s>>>(scratch, nblk, out4);
  return cudaGetLastError();
}

bool device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" elbm_status elbm_reduce_noalloc(const void* pops, const float* scale, const int64_t dims[3],
                                           elbm_precision prec, const double u[3], const elbm_bc* bc,
                                           const float* source, void* cuda_stream, double out4[4]) {
  if (!pops || !dims || !u || !out4) return ELBM_ERR_ARG;
  if ((int)prec < 0 || (int)prec > 3) return ELBM_ERR_ARG;
  if (prec >= ELBM_F32_F16DEV && !scale) return ELBM_ERR_ARG;
  // the kernels read these directly: a host pointer here would make them fault
  if (!device_ptr(pops) || (prec >= ELBM_F32_F16DEV && !device_ptr(scale)) || (source && !device_ptr(source)))
    return ELBM_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 1 || dims[a] > 65535) return ELBM_ERR_ARG;
  const double N = (double)dims[0] * (double)dims[1] * (double)dims[2];
  if (27.0 * N >= 2147483647.0) return ELBM_ERR_ARG;  // same lattice limit as elbm_create
  if (bc && bc->dirichlet_x != 0 && bc->dirichlet_x != 1) return ELBM_ERR_ARG;
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return ELBM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  Grid G{(int)dims[0], (int)dims[1], (int)dims[2], (size_t)N, bc ? bc->dirichlet_x : 0};
  const bool host_out = !device_ptr(out4);
  double* dst = host_out ? scratch + 4 * kMaxPartials : out4;
  cudaError_t e = cudaErrorInvalidValue;
  switch ((int)prec) {
    case 0: e = launch<double>(pops, scale, G, source, u, bc, scratch, dst, s); break;
    case 1: e = launch<float>(pops, scale, G, source, u, bc, scratch, dst, s); break;
    case 2: e = launch<__half>(pops, scale, G, source, u, bc, scratch, dst, s); break;
    case 3: e = launch<__nv_bfloat16>(pops, scale, G, source, u, bc, scratch, dst, s); break;
  }
  if (e != cudaSuccess) return ELBM_ERR_CUDA;
  if (host_out) {
    if (cudaMemcpyAsync(out4, dst, 4 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ELBM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ELBM_ERR_CUDA;
  }
  return ELBM_OK;
}
