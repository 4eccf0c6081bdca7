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

template <typename Elem, int VEL, bool ROOT>
__global__ void __launch_bounds__(256, step_min_blocks<Elem>())
k_step(Field<Elem> in, Elem* __restrict__ pout, float* __restrict__ sout, Grid G,
       const typename Storage<Elem>::real* __restrict__ T6,
       const float* __restrict__ src, const float* __restrict__ u3, int fallback,
       unsigned long long* __restrict__ counters, const PopConsts<typename Storage<Elem>::real> k) {
  using R = typename Storage<Elem>::real;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  bool took = false, proj = false;
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
    if constexpr (VEL == 2) {
      const R un[3] = {R(__ldg(u3 + n)), R(__ldg(u3 + G.N + n)), R(__ldg(u3 + 2 * G.N + n))};
      took = collide_node<R, 2, ROOT>(g, T, k, fallback != 0, phi, un);
    } else {
      took = collide_node<R, VEL, ROOT>(g, T, k, fallback != 0, phi);
    }
    proj = Storage<Elem>::store(pout, sout, G.N, n, g, k.Ek, phi, k.exact_mass != 0);
  }
  // one counter update per block
  const int c = __syncthreads_count(took);
  if (c != 0 && threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(counters, (unsigned long long)c);
  if constexpr (Storage<Elem>::dev) {
    const int p = __syncthreads_count(proj);
    if (p != 0 && threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(counters + 3, (unsigned long long)p);
  }
}

static dim3 block_for(int nx) {
  int bx = nx >= 256 ? 256 : ((nx + 31) / 32) * 32;
  return dim3(bx, 256 / bx, 1);
}

template <typename Elem, int VEL, bool ROOT>
static cudaError_t launch_t(const StepLaunch& L, cudaStream_t s) {
  using R = typename Storage<Elem>::real;
  Field<Elem> in{static_cast<const Elem*>(L.pin), L.sin};
  Grid G{L.nx, L.ny, L.nz, L.N, L.dirichlet};
  dim3 b = block_for(L.nx);
  dim3 g((L.nx + b.x - 1) / b.x, (L.ny + b.y - 1) / b.y, L.nz);
  const PopConsts<R>& k = *reinterpret_cast<const PopConsts<R>*>(std::is_same<R, double>::value ? (const void*)L.kd
                                                                                               : (const void*)L.kf);
  k_step<Elem, VEL, ROOT><<<g, b, 0, s>>>(in, static_cast<Elem*>(L.pout), L.sout, G, static_cast<const R*>(L.T6), L.src,
                                    L.u3, L.fallback, L.counters, k);
  return cudaGetLastError();
}

template <typename Elem>
static cudaError_t launch_v(const StepLaunch& L, cudaStream_t s) {
  // the exact root applies only where u != 0 (kappa = 0 at u = 0)
  const bool root = (std::is_same<Elem, double>::value ? L.kd->root : L.kf->root) != 0;
  if (L.vel == 2) return root ? launch_t<Elem, 2, true>(L, s) : launch_t<Elem, 2, false>(L, s);
  if (L.vel == 1) return root ? launch_t<Elem, 1, true>(L, s) : launch_t<Elem, 1, false>(L, s);
  return launch_t<Elem, 0, false>(L, s);
}

int step_variant(int prec, int nx, int vel, bool root, int requested) {
  if (requested != 0) return requested;
  // auto: the staged-row kernel for the FP32-arithmetic storages with rows of 256 nodes or more
  // (uniform velocity, closed-form stabilizer), else the per-node kernel.  Measured, ms/step
  // per-node -> staged: 256^3 plume FP32 0.684 -> 0.588, BF16 deviations 0.782 -> 0.769, FP16
  // deviations 0.777 -> 0.779 (before the deviation kernels' spill fix); 384^3 heterogeneous
  // (tensor field, source, Dirichlet) FP32 2.83 -> 2.48, FP16 2.88 -> 2.35; 320 x 256 x 256 (row
  // length not compiled in) FP32 0.90 -> 0.72, FP16 1.00 -> 0.85.  Kept on the per-node kernel:
  // rows shorter than a block (192^3: FP32 0.256 vs 0.279, FP16 0.279 vs 0.344), per-node
  // velocity fields (256^3: FP32 1.23 vs 1.65, FP16 1.37 vs 1.77; the per-node tables need the
  // registers the staged kernel's persistent loop holds) and FP64 (arithmetic-bound).
  if (prec != 0 && nx >= 256 && vel != 2 && !root && rows_eligible(prec, nx)) return 2;
  return 1;
}

cudaError_t launch_step(const StepLaunch& L, cudaStream_t s) {
  const bool root = (L.prec == 0 ? L.kd->root : L.kf->root) != 0;
  const int v = step_variant(L.prec, L.nx, L.vel, root, L.variant);
  if (v == 3) return launch_step_pipe(L, s);
  if (v == 2)
    return rows_eligible(L.prec, L.nx) ? launch_step_rows(L, s) : cudaErrorNotSupported;
  switch (L.prec) {
    case 0: return launch_v<double>(L, s);
    case 1: return launch_v<float>(L, s);
    case 2: return launch_v<__half>(L, s);
    case 3: return launch_v<__nv_bfloat16>(L, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace elbm
