// Fused collide-stream kernel: one thread per node pulls its 27 populations,
// collides them in registers (collide.cuh) and writes the 27 post-collision
// values to its own node of the other buffer (coalesced writes, A/B buffers).
#include "internal.h"
#include "pull.cuh"

namespace elbm {

// Resident blocks per SM requested from the register allocator (256 threads each).
#ifndef ELBM_STEP_MINB
#define ELBM_STEP_MINB 3
#endif
template <typename Elem>
constexpr int step_min_blocks() {
  return std::is_same<Elem, double>::value ? 1 : ELBM_STEP_MINB;
}

template <typename Elem, int VEL>
__global__ void __launch_bounds__(256, step_min_blocks<Elem>())
k_step(Field<Elem> in, Elem* __restrict__ pout, float* __restrict__ sout, Grid G,
       const typename Storage<Elem>::real* __restrict__ T6,
       const float* __restrict__ src, int fallback, unsigned long long* __restrict__ counters,
       const PopConsts<typename Storage<Elem>::real> k) {
  using R = typename Storage<Elem>::real;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  bool took = false;
  if (x < G.nx && y < G.ny) {
    const int n = x + G.nx * (y + G.ny * z);
    R g[Q];
    pull_node<Elem, R>(g, in, G, x, y, z, k);
    if (src != nullptr) {
      // merged Strang half-steps of consecutive steps (Section 3.3)
      const R r = k.src_step * R(__ldg(src + n));
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] += r * k.E[i];
    }
    const Sym6<R> T = load_T<R>(T6, G.N, n, k.T);
    R phi;
    took = collide_node<R, VEL>(g, T, k, fallback != 0, phi);
    Storage<Elem>::store(pout, sout, G.N, n, g, k.E, phi);
  }
  const unsigned m = __ballot_sync(0xffffffffu, took);
  if (m != 0u && ((threadIdx.y * blockDim.x + threadIdx.x) & 31) == 0) atomicAdd(counters, (unsigned long long)__popc(m));
}

static dim3 block_for(int nx) {
  int bx = nx >= 256 ? 256 : ((nx + 31) / 32) * 32;
  return dim3(bx, 256 / bx, 1);
}

template <typename Elem, int VEL>
static cudaError_t launch_t(const StepLaunch& L, cudaStream_t s) {
  using R = typename Storage<Elem>::real;
  Field<Elem> in{static_cast<const Elem*>(L.pin), L.sin};
  Grid G{L.nx, L.ny, L.nz, L.N, L.dirichlet};
  dim3 b = block_for(L.nx);
  dim3 g((L.nx + b.x - 1) / b.x, (L.ny + b.y - 1) / b.y, L.nz);
  const PopConsts<R>& k = *reinterpret_cast<const PopConsts<R>*>(std::is_same<R, double>::value ? (const void*)L.kd
                                                                                               : (const void*)L.kf);
  k_step<Elem, VEL><<<g, b, 0, s>>>(in, static_cast<Elem*>(L.pout), L.sout, G, static_cast<const R*>(L.T6), L.src,
                                    L.fallback, L.counters, k);
  return cudaGetLastError();
}

cudaError_t launch_step(const StepLaunch& L, cudaStream_t s) {
  const bool v = L.vel != 0;
  switch (L.prec) {
    case 0: return v ? launch_t<double, 1>(L, s) : launch_t<double, 0>(L, s);
    case 1: return v ? launch_t<float, 1>(L, s) : launch_t<float, 0>(L, s);
    case 2: return v ? launch_t<__half, 1>(L, s) : launch_t<__half, 0>(L, s);
    case 3: return v ? launch_t<__nv_bfloat16, 1>(L, s) : launch_t<__nv_bfloat16, 0>(L, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace elbm
