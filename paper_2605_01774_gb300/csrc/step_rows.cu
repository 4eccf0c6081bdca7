// Fused collide-stream kernel with bulk-asynchronous staging of the pulled rows.
//
// A persistent block takes x-rows (y, z) of the lattice from a row ticket counter.  For
// each row it stages in shared memory, with cp.async.bulk copies completing on an
// mbarrier, the 27 whole source rows the pull needs -- population plane i, row
// (y - c_iy, z - c_iz) -- and, for the deviation storages, the 9 rows of the FP32 scale
// plane.  The periodic x-shift is an index wrap inside the staged row.  STAGES buffers
// rotate: the copies of the next STAGES - 1 rows are in flight while the current row is
// collided, so memory parallelism does not depend on registers, and rows are handed out
// dynamically so that blocks meeting costly rows (positivity fallback) do not set the
// kernel's length.  Collision and store are those of the one-thread-per-node kernel,
// in the same order, so both give bit-equal results.  Requires Nx % 8 == 0 (16-byte
// aligned rows); every wait is bounded.
#include <algorithm>

#include "bulk.cuh"
#include "internal.h"
#include "pull.cuh"

#ifndef ELBM_ROWS_STAGES
#define ELBM_ROWS_STAGES 2
#endif
// Resident 256-thread blocks per SM requested from the register allocator.
#ifndef ELBM_ROWS_MINB
#define ELBM_ROWS_MINB 3
#endif

namespace elbm {

namespace {

// Threads per block: 256, or one thread per node for the compiled-in row length 384.
__host__ __device__ constexpr int block_threads(int WC) { return WC == 384 ? 384 : 256; }
constexpr int STAGES = ELBM_ROWS_STAGES;         // staging buffers per block
constexpr long long WAIT_LIMIT = 2000000000ll;   // clock cycles (about one second)
constexpr int TICKET = 4, DONE = 5;              // counters[] slots of the row scheduler

static_assert(STAGES >= 2 && STAGES <= 4, "2 to 4 staging buffers");

__host__ __device__ constexpr size_t stage_bytes_for(int W, size_t e, bool dev) {
  return 27ull * W * e + (dev ? 9ull * W * sizeof(float) : 0ull);
}

template <typename Elem>
__host__ __device__ constexpr size_t stage_bytes(int W) {
  return stage_bytes_for(W, sizeof(Elem), Storage<Elem>::dev);
}

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Copies of one row of length W, spread over the lanes of warp 0 (lane 0 posts the byte
// count first).
template <typename Elem>
__device__ void issue_row(const Field<Elem>& in, const Grid& G, int W, int row, unsigned char* stage, uint64_t* bar) {
  const int lane = threadIdx.x & 31;
  const int Ny = G.ny, Nz = G.nz;
  const int y = row % Ny, z = row / Ny;
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)stage_bytes<Elem>(W));
  __syncwarp();
  constexpr bool dev = Storage<Elem>::dev;
  Elem* planes = reinterpret_cast<Elem*>(stage);
  float* srows = reinterpret_cast<float*>(stage + 27ull * W * sizeof(Elem));
  for (int c = lane; c < (dev ? 36 : 27); c += 32) {
    if (c < 27) {
      const int ys = wrap(y - cy_of(c), Ny), zs = wrap(z - cz_of(c), Nz);
      bulk_copy_g2s(planes + (size_t)c * W, in.pops + (size_t)c * G.N + (size_t)(ys + Ny * zs) * W,
                    W * sizeof(Elem), bar);
    } else if constexpr (dev) {
      const int r = c - 27;                              // scale row r = 3 (cy + 1) + (cz + 1)
      const int ys = wrap(y - (r / 3 - 1), Ny), zs = wrap(z - (r % 3 - 1), Nz);
      bulk_copy_g2s(srows + (size_t)r * W, in.scale + (size_t)(ys + Ny * zs) * W, W * sizeof(float), bar);
    }
  }
}

// Populations of node x from the staged row: plane i holds source row (y - c_iy, z - c_iz),
// of which node x pulls element x - c_ix (periodic wrap: xm = x - 1, xp = x + 1 mod W).
template <typename Elem, typename R>
__device__ __forceinline__ void staged_pull(R (&g)[Q], const unsigned char* stage, int W, int x, const PopConsts<R>& k) {
  const int xm = x == 0 ? W - 1 : x - 1, xp = x == W - 1 ? 0 : x + 1;
  const Elem* P = reinterpret_cast<const Elem*>(stage);
  if constexpr (Storage<Elem>::dev) {
    const float* S = reinterpret_cast<const float*>(stage + 27ull * W * sizeof(Elem));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int xs = cx_of(i) == 1 ? xm : (cx_of(i) == -1 ? xp : x);
      const float s = S[(i % 9) * W + xs];
      g[i] = s * fmaf(float(1.0 / (1 << qexp_of(i))), Codec<Elem>::to_f(P[i * W + xs]), k.E[i]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int xs = cx_of(i) == 1 ? xm : (cx_of(i) == -1 ? xp : x);
      g[i] = R(P[i * W + xs]);
    }
  }
}

// Halfway anti-bounce-back at the Dirichlet x faces: incoming populations are rebuilt
// from the node's own outgoing ones, read from global memory (Section 2.4).
template <typename Elem, typename R>
__device__ __forceinline__ void abb_faces(R (&g)[Q], const Field<Elem>& f, const Grid& G, int x, int n,
                                          const PopConsts<R>& k) {
  using ST = Storage<Elem>;
  if (x == 0) {
#pragma unroll
    for (int i = 0; i < Q; ++i)
      if (cx_of(i) == 1) g[i] = R(2.0 * w_of(i)) * k.phi_lo - ST::load(f.pops, f.scale, G.N, opp_of(i), n, k.E[opp_of(i)]);
  }
  if (x == G.nx - 1) {
#pragma unroll
    for (int i = 0; i < Q; ++i)
      if (cx_of(i) == -1) g[i] = R(2.0 * w_of(i)) * k.phi_hi - ST::load(f.pops, f.scale, G.N, opp_of(i), n, k.E[opp_of(i)]);
  }
}

// Resident blocks per SM requested from the register allocator: 768 threads for FP32 storage
// types (3 x 256 or 2 x 384), one block for FP64.
template <typename Elem, int WC>
constexpr int rows_min_blocks() {
  return std::is_same<Elem, double>::value ? 1 : (block_threads(WC) == 384 ? 2 : ELBM_ROWS_MINB);
}

}  // namespace

// Next row for this block from the ticket counter (warp 0; the value is warp-uniform), or
// nrows once the counter has run past the last row.
__device__ __forceinline__ int take_row(unsigned long long* counters, int nrows, bool& exhausted) {
  int row = nrows;
  if (!exhausted) {
    unsigned long long t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(counters + TICKET, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t < (unsigned long long)nrows) row = (int)t;
    else exhausted = true;
  }
  return row;
}

// WC > 0: the row length nx as a compile-time constant (shared-memory offsets become
// immediates), else taken from G.
// counters[0]: fallback nodes; [2]: set when a staging wait ran out; [3]: nodes stored as
// their equilibrium shape (deviation storages, see Storage::store); [TICKET]: rows handed
// out in this launch; [DONE]: blocks finished -- the last one resets both for the next launch.
template <typename Elem, int VEL, bool ROOT, int WC>
__global__ void __launch_bounds__(block_threads(WC), rows_min_blocks<Elem, WC>())
k_step_rows(Field<Elem> in, Elem* __restrict__ pout, float* __restrict__ sout, Grid G,
            const typename Storage<Elem>::real* __restrict__ T6, const float* __restrict__ src,
            const float* __restrict__ u3, int fallback, unsigned long long* __restrict__ counters,
            const PopConsts<typename Storage<Elem>::real> k) {
  using R = typename Storage<Elem>::real;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[STAGES];
  __shared__ int s_row[STAGES];
  __shared__ int abort_flag;
  const int W = WC > 0 ? WC : G.nx;
  const size_t SB = stage_bytes<Elem>(W);
  const int nrows = G.ny * G.nz;
  const bool producer = threadIdx.x < 32;     // warp 0 takes the rows and issues their copies
  if (threadIdx.x == 0) {
#pragma unroll
    for (int b = 0; b < STAGES; ++b) mbar_init(&bars[b], 1);
    mbar_fence_init();
    abort_flag = 0;
  }
  __syncthreads();
  bool exhausted = false;
  // thread 0: the ticket of the next row to issue, taken one iteration ahead so that the
  // atomic's round trip overlaps a row of collisions instead of delaying warp 0
  unsigned long long pend = 0;
  if (producer) {
    for (int m = 0; m < STAGES - 1; ++m) {
      const int row = take_row(counters, nrows, exhausted);
      if (threadIdx.x == 0) s_row[m] = row;
      if (row < nrows) issue_row(in, G, W, row, smem + m * SB, &bars[m]);
    }
    if (!exhausted && threadIdx.x == 0) pend = atomicAdd(counters + TICKET, 1ull);
  }
  __syncthreads();
  unsigned took = 0, proj = 0;
  int it = 0;
  for (;; ++it) {
    const int s = it % STAGES;
    const int row = s_row[s];
    if (row >= nrows) break;                  // rows are handed out in increasing order
    if (producer) {
      // the buffer of iteration it + STAGES - 1 was last read in iteration it - 1, which
      // ended with a block barrier
      const int sm = (it + STAGES - 1) % STAGES;
      int nrow = nrows;
      if (!exhausted) {
        const unsigned long long t = __shfl_sync(0xffffffffu, pend, 0);
        if (t < (unsigned long long)nrows) {
          nrow = (int)t;
          if (threadIdx.x == 0) pend = atomicAdd(counters + TICKET, 1ull);
        } else {
          exhausted = true;
        }
      }
      if (threadIdx.x == 0) s_row[sm] = nrow;
      // ordering of the previous reads of this buffer before the copies: the block barrier
      if (nrow < nrows) issue_row(in, G, W, nrow, smem + sm * SB, &bars[sm]);
    }
    if (!mbar_wait_bounded(&bars[s], (it / STAGES) & 1, WAIT_LIMIT)) {
      abort_flag = 1;
    } else {
      const unsigned char* stage = smem + s * SB;
      const size_t row0 = (size_t)row * W;
      for (int x = threadIdx.x; x < W; x += block_threads(WC)) {
        const int n = (int)(row0 + x);
        R g[Q];
        staged_pull<Elem, R>(g, stage, W, x, k);
        if (G.dirichlet) abb_faces<Elem, R>(g, in, G, x, n, k);
        if (src != nullptr) {
          // merged Strang half-steps of consecutive steps (Section 3.3)
          const R r = k.src_step * R(__ldg(src + n));
#pragma unroll
          for (int i = 0; i < Q; ++i) g[i] += r * k.E[i];
        }
        const Sym6<R> T = load_T<R>(T6, G.N, n, k.T);
        R phi;
        bool t;
        if constexpr (VEL == 2) {
          const R un[3] = {R(__ldg(u3 + n)), R(__ldg(u3 + G.N + n)), R(__ldg(u3 + 2 * G.N + n))};
          t = collide_node<R, 2, ROOT>(g, T, k, fallback != 0, phi, un);
        } else {
          t = collide_node<R, VEL, ROOT>(g, T, k, fallback != 0, phi);
        }
        took += t ? 1u : 0u;
        proj += Storage<Elem>::store(pout, sout, (int)G.N, n, g, k.Ek, phi, k.exact_mass != 0) ? 1u : 0u;
      }
    }
    __syncthreads();
    if (abort_flag) break;
  }
  if (abort_flag && threadIdx.x == 0) {
    // leave no copy in flight into this block's shared memory (waits bounded): the buffers
    // hold the rows of iterations it .. it + STAGES - 1, issued where s_row < nrows
    atomicExch(counters + 2, 1ull);
    for (int m = it; m < it + STAGES; ++m)
      if (s_row[m % STAGES] < nrows) mbar_wait_bounded(&bars[m % STAGES], (m / STAGES) & 1, WAIT_LIMIT);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) took += __shfl_xor_sync(0xffffffffu, took, o);
  if (took != 0u && (threadIdx.x & 31) == 0) atomicAdd(counters, (unsigned long long)took);
  if constexpr (Storage<Elem>::dev) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) proj += __shfl_xor_sync(0xffffffffu, proj, o);
    if (proj != 0u && (threadIdx.x & 31) == 0) atomicAdd(counters + 3, (unsigned long long)proj);
  }
  if (threadIdx.x == 0) {
    // every block has taken its last ticket before it counts itself done
    __threadfence();
    if (atomicAdd(counters + DONE, 1ull) == (unsigned long long)gridDim.x - 1) {
      atomicExch(counters + TICKET, 0ull);
      atomicExch(counters + DONE, 0ull);
    }
  }
}

namespace {

// Blocks of k_step_rows<Elem, VEL, ROOT, WC> resident per SM at row length W (0: not
// launchable); raises the kernel's dynamic shared-memory limit as needed.  Cached per
// (device, W).
template <typename Elem, int VEL, bool ROOT, int WC>
int rows_occupancy(int W) {
  static int c_dev = -1, c_w = -1, c_nb = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev == c_dev && W == c_w) return c_nb;
  const size_t dyn = STAGES * stage_bytes<Elem>(W);
  int nb = 0;
  if (cudaFuncSetAttribute(k_step_rows<Elem, VEL, ROOT, WC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) ==
          cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_rows<Elem, VEL, ROOT, WC>, block_threads(WC), dyn) ==
          cudaSuccess) {
    c_dev = dev;
    c_w = W;
    c_nb = nb;
    return nb;
  }
  cudaGetLastError();
  return 0;
}

template <typename Elem, int VEL, bool ROOT, int WC>
cudaError_t launch_rows_t(const StepLaunch& L, cudaStream_t s) {
  using R = typename Storage<Elem>::real;
  const int nb = rows_occupancy<Elem, VEL, ROOT, WC>(L.nx);
  if (nb <= 0) return cudaErrorNotSupported;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long nrows = (long long)L.ny * L.nz;
  const int grid = (int)std::min<long long>(nrows, (long long)nb * nsm);
  Field<Elem> in{static_cast<const Elem*>(L.pin), L.sin};
  Grid G{L.nx, L.ny, L.nz, L.N, L.dirichlet};
  const PopConsts<R>& k = *reinterpret_cast<const PopConsts<R>*>(std::is_same<R, double>::value ? (const void*)L.kd
                                                                                               : (const void*)L.kf);
  k_step_rows<Elem, VEL, ROOT, WC><<<grid, block_threads(WC), STAGES * stage_bytes<Elem>(L.nx), s>>>(
      in, static_cast<Elem*>(L.pout), L.sout, G, static_cast<const R*>(L.T6), L.src, L.u3, L.fallback, L.counters, k);
  return cudaGetLastError();
}

template <typename Elem>
cudaError_t launch_rows_v(const StepLaunch& L, cudaStream_t s) {
  const bool root = (std::is_same<Elem, double>::value ? L.kd->root : L.kf->root) != 0;
  if (L.vel == 2) return root ? launch_rows_t<Elem, 2, true, 0>(L, s) : launch_rows_t<Elem, 2, false, 0>(L, s);
  if (root) return L.vel == 1 ? launch_rows_t<Elem, 1, true, 0>(L, s) : launch_rows_t<Elem, 0, false, 0>(L, s);
  // closed-form stabilizer, uniform velocity: row lengths 256, 384 and 512 compiled in
  if (L.nx == 256) return L.vel == 1 ? launch_rows_t<Elem, 1, false, 256>(L, s) : launch_rows_t<Elem, 0, false, 256>(L, s);
  if (L.nx == 512) return L.vel == 1 ? launch_rows_t<Elem, 1, false, 512>(L, s) : launch_rows_t<Elem, 0, false, 512>(L, s);
  if (L.nx == 384) return L.vel == 1 ? launch_rows_t<Elem, 1, false, 384>(L, s) : launch_rows_t<Elem, 0, false, 384>(L, s);
  return L.vel == 1 ? launch_rows_t<Elem, 1, false, 0>(L, s) : launch_rows_t<Elem, 0, false, 0>(L, s);
}

}  // namespace

// Shared memory of all staging buffers within 200 KiB; rows of 16-byte multiples.
bool rows_eligible(int prec, int nx) {
  if (nx < 8 || nx > 4096 || nx % 8 != 0) return false;
  const size_t e = prec == 0 ? 8 : (prec == 1 ? 4 : 2);
  return STAGES * stage_bytes_for(nx, e, prec >= 2) <= 200 * 1024;
}

cudaError_t launch_step_rows(const StepLaunch& L, cudaStream_t s) {
  if (!rows_eligible(L.prec, L.nx)) return cudaErrorNotSupported;
  switch (L.prec) {
    case 0: return launch_rows_v<double>(L, s);
    case 1: return launch_rows_v<float>(L, s);
    case 2: return launch_rows_v<__half>(L, s);
    case 3: return launch_rows_v<__nv_bfloat16>(L, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace elbm
