// Fused collide-stream kernel with bulk-asynchronous staging of the pulled rows.
//
// A persistent block takes x-rows (y, z) of the lattice from a row ticket counter.  For
// each row it stages in shared memory, with cp.async.bulk copies completing on an
// mbarrier, the 27 whole source rows the pull needs -- population plane i, row
// (y - c_iy, z - c_iz) -- and, for the deviation storages, the 9 rows of the FP32 scale
// plane (with a per-node tensor field or source, also the destination row's T and source
// rows).  The periodic x-shift is an index wrap inside the staged row.  STAGES buffers
// rotate: once every thread has read its nodes' populations of a row into registers (one
// block barrier), the buffer is refilled with the row STAGES ahead before the collisions,
// its copies spread over all warps (one warp issues bulk copies at about one per 80
// cycles), so the next rows' copies are in flight while this one is collided and memory
// parallelism does not depend on registers.  Rows are handed out dynamically so that
// blocks meeting costly rows (positivity fallback, boundary faces) do not set the
// kernel's length.  Collision and store are those of the one-thread-per-node kernel, in
// the same order, so both give bit-equal results.  A second kernel in this file
// (k_step_pipe) replaces the block barrier by a producer warp and full/empty mbarriers
// per stage.  Requires Nx % 8 == 0 (16-byte aligned rows); every wait is bounded.
#include <algorithm>

#include "bulk.cuh"
#include "internal.h"
#include "pull.cuh"

#ifndef ELBM_ROWS_STAGES
#define ELBM_ROWS_STAGES 2
#endif
// Resident 256-thread blocks per SM requested from the register allocator: FP32 storage (80
// registers), deviation storages (64 registers; measured on the 256^3 plume, 0.726 -> 0.701
// ms/step over 600 steps for FP16 with four blocks instead of three).
#ifndef ELBM_ROWS_MINB
#define ELBM_ROWS_MINB 3
#endif
#ifndef ELBM_ROWS_MINB_DEV
#define ELBM_ROWS_MINB_DEV 4
#endif
// 384-thread blocks (row length 384 compiled in) per SM requested from the register allocator
// Shared memory (bytes, all stages) within which the destination row's T-field and source rows
// are staged with the populations (0: read from global memory by each thread)
#ifndef ELBM_ROWS_FIELD_BUDGET
#define ELBM_ROWS_FIELD_BUDGET (200 * 1024)
#endif
#ifndef ELBM_ROWS_MINB_384
#define ELBM_ROWS_MINB_384 2
#endif
#ifndef ELBM_ROWS_MINB_384_DEV
#define ELBM_ROWS_MINB_384_DEV 2
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

// Layout of one stage: the 27 pulled population rows (and, for the deviation storages, the 9
// scale rows), then optionally the destination row's 6 T-field rows and its source row, so that
// the collision reads every per-node input from shared memory.  Offsets 0 = not staged.
struct StageFmt {
  unsigned bytes;     // bytes one row's copies deliver (the expect-tx count)
  unsigned t_off;     // the T rows (6 W values of the arithmetic type), or 0
  unsigned src_off;   // the source row (W floats), or 0
};

template <typename Elem>
StageFmt stage_fmt(int W, bool has_T, bool has_src, size_t budget) {
  using R = typename Storage<Elem>::real;
  StageFmt f{(unsigned)stage_bytes<Elem>(W), 0u, 0u};
  const size_t t = has_T ? 6ull * W * sizeof(R) : 0, r = has_src ? (size_t)W * sizeof(float) : 0;
  if (t + r > 0 && STAGES * (f.bytes + t + r) <= budget) {
    if (has_T) f.t_off = f.bytes;
    if (has_src) f.src_off = f.bytes + (unsigned)t;
    f.bytes += (unsigned)(t + r);
  }
  return f;
}

// Copies of one row of length W: those with index c = first, first + step, ... (the caller
// posts the byte count on the mbarrier, sf.bytes, once per row).
template <typename Elem>
__device__ void issue_copies(const Field<Elem>& in, const Grid& G, int W, int row, unsigned char* stage, uint64_t* bar,
                             const StageFmt& sf, const typename Storage<Elem>::real* T6, const float* src, int first,
                             int step) {
  using R = typename Storage<Elem>::real;
  const int Ny = G.ny, Nz = G.nz;
  const int y = row % Ny, z = row / Ny;
  constexpr bool dev = Storage<Elem>::dev;
  constexpr int nbase = dev ? 36 : 27;
  Elem* planes = reinterpret_cast<Elem*>(stage);
  float* srows = reinterpret_cast<float*>(stage + 27ull * W * sizeof(Elem));
  const int ncopies = nbase + (sf.t_off ? 6 : 0) + (sf.src_off ? 1 : 0);
  for (int c = first; c < ncopies; c += step) {
    if (c < 27) {
      const int ys = wrap(y - cy_of(c), Ny), zs = wrap(z - cz_of(c), Nz);
      bulk_copy_g2s(planes + (size_t)c * W, in.pops + (size_t)c * G.N + (size_t)(ys + Ny * zs) * W,
                    W * sizeof(Elem), bar);
    } else if (dev && c < nbase) {
      const int r = c - 27;                              // scale row r = 3 (cy + 1) + (cz + 1)
      const int ys = wrap(y - (r / 3 - 1), Ny), zs = wrap(z - (r % 3 - 1), Nz);
      bulk_copy_g2s(srows + (size_t)r * W, in.scale + (size_t)(ys + Ny * zs) * W, W * sizeof(float), bar);
    } else if (sf.t_off && c < nbase + 6) {
      const int q = c - nbase;                           // T component q of the destination row
      bulk_copy_g2s(stage + sf.t_off + (size_t)q * W * sizeof(R), T6 + (size_t)q * G.N + (size_t)row * W,
                    W * sizeof(R), bar);
    } else {
      bulk_copy_g2s(stage + sf.src_off, src + (size_t)row * W, W * sizeof(float), bar);
    }
  }
}

// One copy of a row's refill, fixed for the launch: the source plane's first row, the copy's
// offset in the stage, and the row bytes with the (cy, cz) shift of the source row packed in
// `meta` (bits 0-15 bytes, 16-19 cy + 1, 20-23 cz + 1).  Copy c of row (y, z) reads the plane's
// row (y - cy, z - cz), wrapped, as issue_copies does.
struct __align__(16) CopyDesc {
  const unsigned char* plane;
  unsigned dst;
  unsigned meta;
};

template <typename Elem>
__device__ CopyDesc copy_desc(const Field<Elem>& in, const Grid& G, int W, const StageFmt& sf,
                              const typename Storage<Elem>::real* T6, const float* src, int c) {
  using R = typename Storage<Elem>::real;
  constexpr bool dev = Storage<Elem>::dev;
  constexpr int nbase = dev ? 36 : 27;
  const unsigned char* plane;
  unsigned dst, bytes;
  int cy = 0, cz = 0;
  if (c < 27) {
    plane = reinterpret_cast<const unsigned char*>(in.pops + (size_t)c * G.N);
    dst = (unsigned)((size_t)c * W * sizeof(Elem));
    bytes = W * sizeof(Elem);
    cy = cy_of(c);
    cz = cz_of(c);
  } else if (dev && c < nbase) {
    const int r = c - 27;                              // scale row r = 3 (cy + 1) + (cz + 1)
    plane = reinterpret_cast<const unsigned char*>(in.scale);
    dst = (unsigned)(27ull * W * sizeof(Elem) + (size_t)r * W * sizeof(float));
    bytes = W * sizeof(float);
    cy = r / 3 - 1;
    cz = r % 3 - 1;
  } else if (sf.t_off && c < nbase + 6) {
    const int q = c - nbase;                           // T component q of the destination row
    plane = reinterpret_cast<const unsigned char*>(T6 + (size_t)q * G.N);
    dst = sf.t_off + (unsigned)((size_t)q * W * sizeof(R));
    bytes = W * sizeof(R);
  } else {
    plane = reinterpret_cast<const unsigned char*>(src);
    dst = sf.src_off;
    bytes = W * sizeof(float);
  }
  return CopyDesc{plane, dst, bytes | (unsigned)(cy + 1) << 16 | (unsigned)(cz + 1) << 20};
}

// The copy of descriptor d for the row (y, z) (one bulk copy of d's row bytes).
__device__ __forceinline__ void issue_desc(const CopyDesc& d, int y, int z, const Grid& G, unsigned char* stage,
                                           uint64_t* bar) {
  const unsigned bytes = d.meta & 0xffffu;
  const int ys = wrap(y - (int)((d.meta >> 16) & 15u) + 1, G.ny);
  const int zs = wrap(z - (int)((d.meta >> 20) & 15u) + 1, G.nz);
  bulk_copy_g2s(stage + d.dst, d.plane + (size_t)(ys + G.ny * zs) * bytes, bytes, bar);
}

// All copies of one row, spread over the lanes of the calling warp (lane 0 posts the byte count
// first).
template <typename Elem>
__device__ void issue_row(const Field<Elem>& in, const Grid& G, int W, int row, unsigned char* stage, uint64_t* bar,
                          const StageFmt& sf, const typename Storage<Elem>::real* T6, const float* src) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) mbar_arrive_expect_tx(bar, sf.bytes);
  __syncwarp();
  issue_copies(in, G, W, row, stage, bar, sf, T6, src, lane, 32);
}

// Populations of node x from the staged row: plane i holds source row (y - c_iy, z - c_iz),
// of which node x pulls element x - c_ix (periodic wrap: xm = x - 1, xp = x + 1 mod W).
// Es: the equilibrium shape E_i of the deviation storages, a shared-memory copy of the block
// (read afresh in every row: held in registers across the row loop, the 27 values make the
// kernel spill).
template <typename Elem, typename R>
__device__ __forceinline__ void staged_pull(R (&g)[Q], const unsigned char* stage, int W, int x, const float* Es) {
  const int xm = x == 0 ? W - 1 : x - 1, xp = x == W - 1 ? 0 : x + 1;
  const Elem* P = reinterpret_cast<const Elem*>(stage);
  if constexpr (Storage<Elem>::dev) {
    const float* S = reinterpret_cast<const float*>(stage + 27ull * W * sizeof(Elem));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int xs = cx_of(i) == 1 ? xm : (cx_of(i) == -1 ? xp : x);
      const float s = S[(i % 9) * W + xs];
      g[i] = s * Codec<Elem>::fma_pow2(P[i * W + xs], qexp_of(i), Es[i]);
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
// types (3 x 256 or 2 x 384), 4 x 256 for the deviation storages at the compiled-in row length
// 256 or 512 (the velocity-field and exact-root kernels keep 3: their per-node tables need the
// registers), one block for FP64.
template <typename Elem, int WC>
constexpr int rows_min_blocks() {
  return std::is_same<Elem, double>::value
             ? 1
             : (block_threads(WC) == 384 ? (Storage<Elem>::dev ? ELBM_ROWS_MINB_384_DEV : ELBM_ROWS_MINB_384)
                                          : (Storage<Elem>::dev && WC > 0 ? ELBM_ROWS_MINB_DEV : ELBM_ROWS_MINB));
}

}  // namespace

// Next row for this block from the ticket counter (one warp; the value is warp-uniform), or
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
            long long wait_limit, int withheld, StageFmt sf, const PopConsts<typename Storage<Elem>::real> k) {
  using R = typename Storage<Elem>::real;
  constexpr int BT = block_threads(WC), NW = BT / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[STAGES];           // completes when a stage's copies have landed
  __shared__ int s_row[STAGES];               // row staged in each buffer (nrows: none)
  __shared__ int s_next[2];                   // row of the refill of iteration it (parity it & 1)
  __shared__ int2 s_nyz[2];                   // its (y, z)
  __shared__ float sE[Q];                     // E_i for the deviation decode (ordered by the first barrier)
  __shared__ CopyDesc s_desc[48];             // the refill's copies (ordered by the first barrier)
  if (threadIdx.x < Q) sE[threadIdx.x] = float(k.E[threadIdx.x]);
  const int W = WC > 0 ? WC : G.nx;
  const int ncopies = (Storage<Elem>::dev ? 36 : 27) + (sf.t_off ? 6 : 0) + (sf.src_off ? 1 : 0);
  if (threadIdx.x < ncopies) s_desc[threadIdx.x] = copy_desc(in, G, W, sf, T6, src, threadIdx.x);
  const size_t SB = sf.bytes;
  const int nrows = G.ny * G.nz;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int b = 0; b < STAGES; ++b) mbar_init(&full[b], 1 + withheld);   // withheld: test hook
    mbar_fence_init();
  }
  __syncthreads();
  // thread 0: the ticket of the next row to issue, taken one row ahead so that the atomic's
  // round trip overlaps a row of collisions
  unsigned long long pend = 0;
  if (warp == 0) {
    bool exhausted = false;
    for (int m = 0; m < STAGES; ++m) {
      const int row = take_row(counters, nrows, exhausted);
      if (lane == 0) s_row[m] = row;
      if (row < nrows) issue_row(in, G, W, row, smem + m * SB, &full[m], sf, T6, src);
    }
    pend = exhausted ? (unsigned long long)nrows : 0ull;
    if (!exhausted && lane == 0) pend = atomicAdd(counters + TICKET, 1ull);
  }
  __syncthreads();
  unsigned took = 0, proj = 0;
  const int nper = (W + BT - 1) / BT;         // nodes of a row per thread (block-uniform)
  // the copies of a refill are spread over all warps, so that no warp issues more than a few
  // (one warp issues bulk copies at about one per 80 cycles)
  const int cfirst = lane * NW + warp;
  int it = 0;
  bool stop = false;
  for (; !stop; ++it) {
    const int s = it % STAGES;
    const int row = s_row[s];
    if (row >= nrows) break;                  // rows are handed out in increasing order
    const bool ok = mbar_wait_bounded(&full[s], (it / STAGES) & 1, wait_limit);
    const unsigned char* stage = smem + s * SB;
    const size_t row0 = (size_t)row * W;
    for (int m = 0; m < nper; ++m) {
      // threads past the end of the row read (and then drop) its last node, so that the pull is
      // unconditional: a conditional pull makes the compiler spill the populations
      const bool valid = ok && threadIdx.x + m * BT < W;
      const int x = min(threadIdx.x + m * BT, W - 1);
      const int n = (int)(row0 + x);
      R g[Q];
      staged_pull<Elem, R>(g, stage, W, x, sE);
      Sym6<R> T;
      if (sf.t_off) {
        const R* Ts = reinterpret_cast<const R*>(stage + sf.t_off);
        T = Sym6<R>{Ts[x], Ts[W + x], Ts[2 * W + x], Ts[3 * W + x], Ts[4 * W + x], Ts[5 * W + x]};
      } else {
        T = load_T<R>(T6, G.N, n, k.T);
      }
      float sv = 0.f;
      if (src != nullptr) sv = sf.src_off ? reinterpret_cast<const float*>(stage + sf.src_off)[x] : __ldg(src + n);
      if (m == nper - 1) {
        // every thread has read the stage of this row into registers: it is refilled with the
        // row of iteration it + STAGES before the collisions, so that STAGES rows are in flight
        // while this one is collided (the block barrier orders the generic reads of the buffer
        // before the copies into it).  Thread 0 publishes the row and posts the byte count for
        // the refill before the barrier (this phase of the buffer has completed: its wait
        // succeeded); the same barrier tells every thread whether a wait of this row ran out,
        // so that the whole block leaves together.
        if (threadIdx.x == 0) {
          const int nrow = pend < (unsigned long long)nrows ? (int)pend : nrows;
          s_next[it & 1] = nrow;
          s_nyz[it & 1] = make_int2(nrow % G.ny, nrow / G.ny);
          if (ok && nrow < nrows) mbar_arrive_expect_tx(&full[s], sf.bytes);
        }
        if (__syncthreads_or(ok ? 0 : 1)) {
          stop = true;
          break;
        }
        const int nrow = s_next[it & 1];
        if (threadIdx.x == 0) {
          s_row[s] = nrow;
          if (nrow < nrows) pend = atomicAdd(counters + TICKET, 1ull);
        }
        // this thread's copy of the refill (the same copy in every row, one per thread at most:
        // ncopies <= 43 < BT), from its launch-long descriptor
        if (nrow < nrows && cfirst < ncopies) {
          const int2 yz = s_nyz[it & 1];
          issue_desc(s_desc[cfirst], yz.x, yz.y, G, smem + s * SB, &full[s]);
        }
      }
      if (!valid) continue;
      if (G.dirichlet) abb_faces<Elem, R>(g, in, G, x, n, k);
      if (src != nullptr) {
        // merged Strang half-steps of consecutive steps (Section 3.3)
        const R r = k.src_step * R(sv);
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] += r * k.E[i];
      }
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
  if (stop) --it;                             // the aborted iteration
  if (stop && threadIdx.x == 0) {
    // leave no copy in flight into this block's shared memory (waits bounded): the buffers
    // hold the rows of iterations it .. it + STAGES - 1, issued where s_row < nrows
    atomicExch(counters + 2, 1ull);
    for (int m = it; m < it + STAGES; ++m)
      if (s_row[m % STAGES] < nrows) {
        for (int w = 0; w < withheld; ++w) mbar_arrive(&full[m % STAGES]);   // the arrivals the test withheld
        mbar_wait_bounded(&full[m % STAGES], (m / STAGES) & 1, WAIT_LIMIT);
      }
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

// ------------------------------------------------------------------------------------------
// Pipelined variant: persistent blocks (two per SM, one for FP64), each a producer warp and NC
// consumer warps sharing a ring of NS row stages.  Stage s carries two mbarriers: full[s] completes when the
// producer's bulk copies of a row have landed (transaction count), empty[s] when every consumer
// lane that worked on that row has arrived.  The unit of consumer work is a 32-node segment of
// a staged row, taken from a shared counter in row order; a lane releases the stage as soon as
// its 27 pulled populations are in registers, before the collision, so a warp that meets costly
// nodes (positivity fallback) holds no stage while it computes and the other warps go on with
// the next segments; there is no block-wide barrier in the loop.  The producer takes rows
// from the same global ticket counter as the per-row kernel, waits for empty[s], and refills.
// When the tickets run out it publishes NS sentinel rows (row index = nrows) so that every
// consumer, whatever segment it took, sees one and leaves.
//
// Correctness conditions (checked on the host, pipe_stages): NC <= NS * nseg, so a consumer can
// never take a segment of row slot k before slot k - NS has completed (that would need more
// than NC segments outstanding) -- the parity of full[s] is therefore unambiguous; NS >= 3.
// The partial per-warp segment (nx % 32 != 0) has idle lanes, which still arrive on empty[s].
// Consumer warps per block of the pipelined kernel: FP32 storage, deviation storages (two
// blocks per SM: 2 x 12 warps at 80 registers, 2 x 10 warps at 96 registers).
#ifndef ELBM_PIPE_NC
#define ELBM_PIPE_NC 11
#endif
#ifndef ELBM_PIPE_NC_DEV
#define ELBM_PIPE_NC_DEV 9
#endif
// Rows handed to a producer per ticket: one global atomic per chunk (the next chunk's ticket
// is taken one chunk ahead), at the cost of up to a chunk of imbalance at the end of a step.
#ifndef ELBM_PIPE_CHUNK
#define ELBM_PIPE_CHUNK 4
#endif
constexpr int PIPE_CHUNK = ELBM_PIPE_CHUNK;
// Resident blocks (independent producer/consumer pipelines) per SM for the FP32-arithmetic
// storages; FP64 runs one.  Measured on the 256^3 plume: one pipeline per SM is limited by the
// rate at which its single producer warp takes rows and issues their copies (FP32 0.71-0.79
// ms/step against 0.52-0.58 for the per-row kernel); two pipelines match the per-row kernel.
#ifndef ELBM_PIPE_BLOCKS
#define ELBM_PIPE_BLOCKS 2
#endif
constexpr int PIPE_MAX_STAGES = 8;
#ifndef ELBM_PIPE_SMEM_KB
#define ELBM_PIPE_SMEM_KB 200
#endif
constexpr size_t PIPE_SMEM_SM = ELBM_PIPE_SMEM_KB * 1024;   // stage rings of all blocks of an SM

__host__ __device__ constexpr int pipe_blocks_for(int prec) { return prec == 0 ? 1 : ELBM_PIPE_BLOCKS; }
template <typename Elem>
__host__ __device__ constexpr int pipe_blocks() {
  return std::is_same<Elem, double>::value ? 1 : ELBM_PIPE_BLOCKS;
}

template <typename Elem, int VEL, bool ROOT>
__host__ __device__ constexpr int pipe_consumer_warps() {
  return std::is_same<Elem, double>::value ? 12
                                            : ((VEL == 2 || ROOT) ? 7 : (Storage<Elem>::dev ? ELBM_PIPE_NC_DEV : ELBM_PIPE_NC));
}

template <typename Elem, int VEL, bool ROOT>
__host__ __device__ constexpr int pipe_threads() {
  return 32 * (pipe_consumer_warps<Elem, VEL, ROOT>() + 1);
}

template <typename Elem, int VEL, bool ROOT, int WC>
__global__ void __launch_bounds__(pipe_threads<Elem, VEL, ROOT>(), pipe_blocks<Elem>())
k_step_pipe(Field<Elem> in, Elem* __restrict__ pout, float* __restrict__ sout, Grid G,
            const typename Storage<Elem>::real* __restrict__ T6, const float* __restrict__ src,
            const float* __restrict__ u3, int fallback, unsigned long long* __restrict__ counters,
            long long wait_limit, int NS, const PopConsts<typename Storage<Elem>::real> k) {
  using R = typename Storage<Elem>::real;
  constexpr int NC = pipe_consumer_warps<Elem, VEL, ROOT>();
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[PIPE_MAX_STAGES], empty[PIPE_MAX_STAGES];
  __shared__ int s_row[PIPE_MAX_STAGES];
  __shared__ int s_item;
  __shared__ int abort_flag;
  __shared__ float sE[Q];                     // E_i for the deviation decode (ordered by the first barrier)
  if (threadIdx.x < Q) sE[threadIdx.x] = float(k.E[threadIdx.x]);
  const int W = WC > 0 ? WC : G.nx;
  const int nseg = (W + 31) >> 5;
  const size_t SB = stage_bytes<Elem>(W);
  const int nrows = G.ny * G.nz;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int b = 0; b < NS; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], 32 * nseg);
    }
    mbar_fence_init();
    s_item = 0;
    abort_flag = 0;
  }
  __syncthreads();
  volatile int* vabort = &abort_flag;

  if (warp == NC) {
    // ---- producer warp
    bool exhausted = false, aborted = false;
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(counters + TICKET, (unsigned long long)PIPE_CHUNK);   // next chunk
    int kk = 0, k_real = 0, sentinels = 0, next_row = 0, left = 0;
    for (; sentinels < NS; ++kk) {
      const int s = kk % NS;
      int row = nrows;
      if (!exhausted && left == 0) {
        const unsigned long long tt = __shfl_sync(0xffffffffu, t, 0);
        if (tt < (unsigned long long)nrows) {
          next_row = (int)tt;
          left = min(PIPE_CHUNK, nrows - next_row);
          if (lane == 0) t = atomicAdd(counters + TICKET, (unsigned long long)PIPE_CHUNK);  // overlaps the rows
        } else {
          exhausted = true;
        }
      }
      if (!exhausted) {
        row = next_row++;
        --left;
      }
      // stage s was last used by slot kk - NS: every consumer lane of that row must have left it
      if (kk >= NS && !mbar_wait_or_abort(&empty[s], ((kk / NS) - 1) & 1, wait_limit, vabort)) {
        aborted = true;
        break;
      }
      if (*vabort) {
        aborted = true;
        break;
      }
      if (lane == 0) s_row[s] = row;             // released by the arrival on full[s]
      if (row < nrows) {
        issue_row(in, G, W, row, smem + s * SB, &full[s], StageFmt{(unsigned)SB, 0u, 0u}, T6, src);
        k_real = kk + 1;
      } else {
        if (lane == 0) mbar_arrive(&full[s]);
        ++sentinels;
      }
    }
    if (aborted) {
      if (lane == 0) {
        *vabort = 1;
        atomicExch(counters + 2, 1ull);
      }
      // no copy may still be writing this block's shared memory when it exits: wait (bounded,
      // full limit) for the row slots issued last whose stages were never refilled
      for (int m = kk - NS > 0 ? kk - NS : 0; m < k_real; ++m)
        mbar_wait_bounded(&full[m % NS], (m / NS) & 1, WAIT_LIMIT);
    }
    if (lane == 0) {
      // this block takes no more tickets; the last block to finish resets the scheduler
      __threadfence();
      if (atomicAdd(counters + DONE, 1ull) == (unsigned long long)gridDim.x - 1) {
        atomicExch(counters + TICKET, 0ull);
        atomicExch(counters + DONE, 0ull);
      }
    }
    return;
  }

  // ---- consumer warps
  unsigned took = 0, proj = 0;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(&s_item, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    const int slot = it / nseg, q = it - slot * nseg, s = slot % NS;
    if (!mbar_wait_or_abort(&full[s], (slot / NS) & 1, wait_limit, vabort)) {
      if (lane == 0 && atomicExch(&abort_flag, 1) == 0) atomicExch(counters + 2, 1ull);
      break;
    }
    const int row = *(volatile int*)&s_row[s];
    if (row >= nrows) break;
    const int x = (q << 5) + lane;
    R g[Q];
    if (x < W) staged_pull<Elem, R>(g, smem + s * SB, W, x, sE);
    // the lane's populations are in registers: release the stage before the collision, so a
    // slow segment holds its stage only for its loads (the arrival orders them before any
    // later copy into the stage)
    mbar_arrive(&empty[s]);
    if (x < W) {
      const int n = row * W + x;
      if (G.dirichlet) abb_faces<Elem, R>(g, in, G, x, n, k);
      if (src != nullptr) {
        // merged Strang half-steps of consecutive steps (Section 3.3)
        const R r = k.src_step * R(__ldg(src + n));
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] += r * k.E[i];
      }
      const Sym6<R> T = load_T<R>(T6, G.N, n, k.T);
      R phi;
      bool tk;
      if constexpr (VEL == 2) {
        const R un[3] = {R(__ldg(u3 + n)), R(__ldg(u3 + G.N + n)), R(__ldg(u3 + 2 * G.N + n))};
        tk = collide_node<R, 2, ROOT>(g, T, k, fallback != 0, phi, un);
      } else {
        tk = collide_node<R, VEL, ROOT>(g, T, k, fallback != 0, phi);
      }
      took += tk ? 1u : 0u;
      proj += Storage<Elem>::store(pout, sout, (int)G.N, n, g, k.Ek, phi, k.exact_mass != 0) ? 1u : 0u;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) took += __shfl_xor_sync(0xffffffffu, took, o);
  if (took != 0u && lane == 0) atomicAdd(counters, (unsigned long long)took);
  if constexpr (Storage<Elem>::dev) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) proj += __shfl_xor_sync(0xffffffffu, proj, o);
    if (proj != 0u && lane == 0) atomicAdd(counters + 3, (unsigned long long)proj);
  }
}

namespace {

// Blocks of k_step_rows<Elem, VEL, ROOT, WC> resident per SM with `dyn` bytes of stages (0: not
// launchable); raises the kernel's dynamic shared-memory limit as needed.  Cached per (device, dyn).
template <typename Elem, int VEL, bool ROOT, int WC>
int rows_occupancy(size_t dyn) {
  static int c_dev[4] = {-1, -1, -1, -1}, c_nb[4] = {0, 0, 0, 0};
  static size_t c_dyn[4] = {0, 0, 0, 0};
  static int next = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  for (int e = 0; e < 4; ++e)
    if (c_dev[e] == dev && c_dyn[e] == dyn) return c_nb[e];
  int nb = 0;
  // raise (never lower) the kernel's limit: another layout may already have been launched
  cudaFuncAttributes fa;
  const int cur = cudaFuncGetAttributes(&fa, k_step_rows<Elem, VEL, ROOT, WC>) == cudaSuccess
                      ? fa.maxDynamicSharedSizeBytes : 0;
  if ((cur >= (int)dyn || cudaFuncSetAttribute(k_step_rows<Elem, VEL, ROOT, WC>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) == cudaSuccess) &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_rows<Elem, VEL, ROOT, WC>, block_threads(WC), dyn) ==
          cudaSuccess) {
    c_dev[next] = dev;
    c_dyn[next] = dyn;
    c_nb[next] = nb;
    next = (next + 1) % 4;
    return nb;
  }
  cudaGetLastError();
  return 0;
}

template <typename Elem, int VEL, bool ROOT, int WC>
cudaError_t launch_rows_t(const StepLaunch& L, cudaStream_t s) {
  using R = typename Storage<Elem>::real;
  // stage the T-field and source rows too where that keeps the resident blocks per SM
  const StageFmt base = stage_fmt<Elem>(L.nx, false, false, 0);
  StageFmt sf = stage_fmt<Elem>(L.nx, L.T6 != nullptr, L.src != nullptr, ELBM_ROWS_FIELD_BUDGET);
  int nb = rows_occupancy<Elem, VEL, ROOT, WC>(STAGES * (size_t)base.bytes);
  if (sf.bytes != base.bytes) {
    const int nbf = rows_occupancy<Elem, VEL, ROOT, WC>(STAGES * (size_t)sf.bytes);
    if (nbf >= nb && nbf > 0) nb = nbf;
    else sf = base;
  }
  if (nb <= 0) return cudaErrorNotSupported;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  // the kernel's shared-memory limit only ever grows (rows_occupancy raised it for both layouts);
  // raise it here only if this launch needs more, so that steps do not change a kernel attribute
  static int c_dev = -1;
  static size_t c_max = 0;
  const size_t dyn = STAGES * (size_t)sf.bytes;
  if (dev != c_dev || dyn > c_max) {
    if (cudaFuncSetAttribute(k_step_rows<Elem, VEL, ROOT, WC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max(dyn, dev == c_dev ? c_max : (size_t)0)) != cudaSuccess)
      return cudaGetLastError();
    c_max = std::max(dyn, dev == c_dev ? c_max : (size_t)0);
    c_dev = dev;
  }
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long nrows = (long long)L.ny * L.nz;
  const int grid = (int)std::min<long long>(nrows, (long long)nb * nsm);
  Field<Elem> in{static_cast<const Elem*>(L.pin), L.sin};
  Grid G{L.nx, L.ny, L.nz, L.N, L.dirichlet};
  const PopConsts<R>& k = *reinterpret_cast<const PopConsts<R>*>(std::is_same<R, double>::value ? (const void*)L.kd
                                                                                               : (const void*)L.kf);
  k_step_rows<Elem, VEL, ROOT, WC><<<grid, block_threads(WC), STAGES * (size_t)sf.bytes, s>>>(
      in, static_cast<Elem*>(L.pout), L.sout, G, static_cast<const R*>(L.T6), L.src, L.u3, L.fallback, L.counters,
      L.wait_limit > 0 ? L.wait_limit : WAIT_LIMIT, L.withheld, sf, k);
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

// ---- pipelined variant: launch configuration

namespace {

// Stages of the pipelined kernel for storage `prec` at row length W (0: not available):
// as many as fit in PIPE_SMEM, at most PIPE_MAX_STAGES, at least 3, and enough that the NC
// consumer warps can never reach a stage two uses ahead (NC <= NS * nseg).
int pipe_stages_for(int prec, int W, int nc) {
  if (W < 8 || W % 8 != 0) return 0;
  const size_t e = prec == 0 ? 8 : (prec == 1 ? 4 : 2);
  const size_t sb = stage_bytes_for(W, e, prec >= 2);
  const int ns = (int)std::min<size_t>(PIPE_MAX_STAGES, PIPE_SMEM_SM / pipe_blocks_for(prec) / sb);
  const int nseg = (W + 31) / 32;
  if (ns < 3 || nc > ns * nseg) return 0;
  return ns;
}

template <typename Elem, int VEL, bool ROOT, int WC>
cudaError_t launch_pipe_t(const StepLaunch& L, cudaStream_t s) {
  using R = typename Storage<Elem>::real;
  constexpr int NC = pipe_consumer_warps<Elem, VEL, ROOT>();
  const int ns = pipe_stages_for(L.prec, L.nx, NC);
  if (ns == 0) return cudaErrorNotSupported;
  const size_t dyn = (size_t)ns * stage_bytes<Elem>(L.nx);
  static int c_dev = -1;
  static size_t c_dyn = 0;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  if (dev != c_dev || dyn > c_dyn) {
    cudaError_t e = cudaFuncSetAttribute(k_step_pipe<Elem, VEL, ROOT, WC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    c_dev = dev;
    c_dyn = dyn;
  }
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long nrows = (long long)L.ny * L.nz;
  const int grid = (int)std::min<long long>(nrows, (long long)pipe_blocks<Elem>() * nsm);
  Field<Elem> in{static_cast<const Elem*>(L.pin), L.sin};
  Grid G{L.nx, L.ny, L.nz, L.N, L.dirichlet};
  const PopConsts<R>& k = *reinterpret_cast<const PopConsts<R>*>(std::is_same<R, double>::value ? (const void*)L.kd
                                                                                               : (const void*)L.kf);
  k_step_pipe<Elem, VEL, ROOT, WC><<<grid, pipe_threads<Elem, VEL, ROOT>(), dyn, s>>>(
      in, static_cast<Elem*>(L.pout), L.sout, G, static_cast<const R*>(L.T6), L.src, L.u3, L.fallback, L.counters,
      L.wait_limit > 0 ? L.wait_limit : WAIT_LIMIT, ns, k);
  return cudaGetLastError();
}

template <typename Elem>
cudaError_t launch_pipe_v(const StepLaunch& L, cudaStream_t s) {
  const bool root = (std::is_same<Elem, double>::value ? L.kd->root : L.kf->root) != 0;
  if (L.vel == 2) return root ? launch_pipe_t<Elem, 2, true, 0>(L, s) : launch_pipe_t<Elem, 2, false, 0>(L, s);
  if (root) return L.vel == 1 ? launch_pipe_t<Elem, 1, true, 0>(L, s) : launch_pipe_t<Elem, 0, false, 0>(L, s);
  // closed-form stabilizer, uniform velocity: row lengths 256, 384 and 512 compiled in
  if (L.nx == 256) return L.vel == 1 ? launch_pipe_t<Elem, 1, false, 256>(L, s) : launch_pipe_t<Elem, 0, false, 256>(L, s);
  if (L.nx == 512) return L.vel == 1 ? launch_pipe_t<Elem, 1, false, 512>(L, s) : launch_pipe_t<Elem, 0, false, 512>(L, s);
  if (L.nx == 384) return L.vel == 1 ? launch_pipe_t<Elem, 1, false, 384>(L, s) : launch_pipe_t<Elem, 0, false, 384>(L, s);
  return L.vel == 1 ? launch_pipe_t<Elem, 1, false, 0>(L, s) : launch_pipe_t<Elem, 0, false, 0>(L, s);
}

}  // namespace

bool pipe_eligible(int prec, int nx, int vel, bool root) {
  int nc = prec >= 2 ? ELBM_PIPE_NC_DEV : ELBM_PIPE_NC;
  if (prec == 0) nc = 12;
  else if (vel == 2 || root) nc = 7;
  return pipe_stages_for(prec, nx, nc) > 0;
}

cudaError_t launch_step_pipe(const StepLaunch& L, cudaStream_t s) {
  const bool root = (L.prec == 0 ? L.kd->root : L.kf->root) != 0;
  if (!pipe_eligible(L.prec, L.nx, L.vel, root)) return cudaErrorNotSupported;
  switch (L.prec) {
    case 0: return launch_pipe_v<double>(L, s);
    case 1: return launch_pipe_v<float>(L, s);
    case 2: return launch_pipe_v<__half>(L, s);
    case 3: return launch_pipe_v<__nv_bfloat16>(L, s);
  }
  return cudaErrorInvalidValue;
}

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
