// Many independent periodic lattices (an orientation / anisotropy sweep) stepped
// together.  Every domain is a cube of edge n_d with its own uniform tensor, zero
// velocity, FP32 populations; its 27 planes are stored contiguously
// [domain][27][n_d^3].  Work is cut into tiles of `tile` consecutive nodes of one
// domain; a tile table maps a global tile index to (domain, first node).
//
//   mode 0  one persistent cooperative kernel runs all steps: blocks take tiles
//           round-robin, then meet at a bounded grid barrier before the next step;
//           the launch is captured once into a CUDA graph.
//   mode 1  one launch per step over all tiles, the step sequence captured in a graph.
//   mode 2  one plain launch of the single-lattice kernel per domain per step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/elbm.h"
#include "../../include/elbm_batch.h"
#include "internal.h"
#include "pull.cuh"

using namespace elbm;

namespace {

struct DomainInfo {
  long long off;   // first node of the domain in the concatenated node space
  int n;           // edge
  float inv_n;     // 1/n (node index decomposition)
  float T[6];      // T = 2I - S (xx, xy, xz, yy, yz, zz)
};

struct BatchArgs {
  const DomainInfo* dom;
  const int* tile_dom;          // tile -> domain
  const int* tile_first;        // tile -> first local node
  int ntiles;
  float* bufA;
  float* bufB;
  unsigned long long* fb_count;
  float eps;
  int fallback;
};

// exact i / n for 0 <= i < 2^24 and n <= 2^12 using a float reciprocal and one correction
__device__ __forceinline__ int div_small(int i, int n, float inv) {
  int q = (int)((float)i * inv);
  const int r = i - q * n;
  q += (r >= n) - (r < 0);
  return q;
}

__device__ __forceinline__ bool batch_node(const BatchArgs& a, const float* __restrict__ in, float* __restrict__ out,
                                           const DomainInfo& d, int local) {
  const int n = d.n;
  const int N = n * n * n;
  const int z = div_small(local, n * n, d.inv_n * d.inv_n);
  const int rem = local - z * n * n;
  const int y = div_small(rem, n, d.inv_n);
  const int x = rem - y * n;
  const float* p = in + 27ll * d.off;
  float* q = out + 27ll * d.off;
  Field<float> f{p, nullptr};
  Grid G{n, n, n, (size_t)N, 0};
  PopConsts<float> k;  // only E (u = 0: W_i) is read by the pull for plain storage
#pragma unroll
  for (int i = 0; i < Q; ++i) k.E[i] = float(w_of(i));
  float g[Q];
  pull_node<float, float>(g, f, G, x, y, z, k);
  const Sym6<float> T{d.T[0], d.T[1], d.T[2], d.T[3], d.T[4], d.T[5]};
  k.eps = a.eps;
  float phi;
  const bool took = collide_node<float, 0>(g, T, k, a.fallback != 0, phi);
#pragma unroll
  for (int i = 0; i < Q; ++i) q[i * N + local] = g[i];
  return took;
}

__device__ __forceinline__ void count_fallback(const BatchArgs& a, bool took) {
  const unsigned m = __ballot_sync(0xffffffffu, took);
  if (m != 0u && (threadIdx.x & 31) == 0) atomicAdd(a.fb_count, (unsigned long long)__popc(m));
}

__device__ __forceinline__ void do_tile(const BatchArgs& a, const float* in, float* out, int t) {
  const DomainInfo& d = a.dom[a.tile_dom[t]];
  const int local = a.tile_first[t] + threadIdx.x;
  bool took = false;
  if (local < d.n * d.n * d.n) took = batch_node(a, in, out, d, local);
  count_fallback(a, took);
}

// Resident 256-thread blocks per SM requested from the register allocator (0: no request; 4
// forces 64 registers and spills, measured slower on the 512-domain sweep).
#ifndef ELBM_BATCH_MINB
#define ELBM_BATCH_MINB 0
#endif

// mode 1: one block per tile
__global__ void __launch_bounds__(256, ELBM_BATCH_MINB) k_batch_step(BatchArgs a, int parity) {
  const float* in = parity ? a.bufB : a.bufA;
  float* out = parity ? a.bufA : a.bufB;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) do_tile(a, in, out, t);
}

// Bounded grid barrier: the last block to arrive advances the generation; the
// others wait for it at most `limit` clock cycles, then set *err and return false.
__device__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned expected, long long limit, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = atomicAdd(gen, 0u);
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u);
    if (arrived == expected - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const long long t0 = clock64();
      while (atomicAdd(gen, 0u) == g) {
        if (atomicAdd(err, 0) != 0 || clock64() - t0 > limit) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// mode 0: persistent kernel, all steps in one launch
__global__ void __launch_bounds__(256, ELBM_BATCH_MINB) k_batch_persistent(BatchArgs a, int nsteps, int parity0, unsigned* bar,
                                                          unsigned expected, long long limit, int* err) {
  int parity = parity0;
  for (int s = 0; s < nsteps; ++s) {
    const float* in = parity ? a.bufB : a.bufA;
    float* out = parity ? a.bufA : a.bufB;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) do_tile(a, in, out, t);
    if (!grid_barrier(bar, bar + 1, expected, limit, err)) return;
    parity ^= 1;
  }
}

__global__ void k_batch_write(const DomainInfo* dom, const int* tile_dom, const int* tile_first, int ntiles,
                              const float* __restrict__ phi0, float* __restrict__ buf) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const DomainInfo d = dom[tile_dom[t]];
    const int local = tile_first[t] + threadIdx.x;
    const int n = d.n, N = n * n * n;
    if (local >= N) continue;
    const int z = div_small(local, n * n, d.inv_n * d.inv_n);
    const int rem = local - z * n * n;
    const int y = div_small(rem, n, d.inv_n);
    const int x = rem - y * n;
    // equilibrium at u = 0 written so that the next pull sees g_i(x) = W_i phi0(x)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int sx = (x + cx_of(i) + n) % n, sy = (y + cy_of(i) + n) % n, sz = (z + cz_of(i) + n) % n;
      buf[27ll * d.off + (long long)i * N + local] = float(w_of(i)) * phi0[d.off + sx + n * (sy + n * sz)];
    }
  }
}

__global__ void k_batch_read(const DomainInfo* dom, const int* tile_dom, const int* tile_first, int ntiles,
                             const float* __restrict__ buf, float* __restrict__ phi, float* __restrict__ pops,
                             int only_dom) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int di = tile_dom[t];
    if (only_dom >= 0 && di != only_dom) continue;
    const DomainInfo d = dom[di];
    const int local = tile_first[t] + threadIdx.x;
    const int n = d.n, N = n * n * n;
    if (local >= N) continue;
    const int z = div_small(local, n * n, d.inv_n * d.inv_n);
    const int rem = local - z * n * n;
    const int y = div_small(rem, n, d.inv_n);
    const int x = rem - y * n;
    Field<float> f{buf + 27ll * d.off, nullptr};
    Grid G{n, n, n, (size_t)N, 0};
    PopConsts<float> k;
#pragma unroll
    for (int i = 0; i < Q; ++i) k.E[i] = float(w_of(i));
    float g[Q];
    pull_node<float, float>(g, f, G, x, y, z, k);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) s += g[i];
    if (phi) phi[d.off + local] = s;
    if (pops) {
#pragma unroll
      for (int i = 0; i < Q; ++i) pops[(long long)i * N + local] = g[i];
    }
  }
}

}  // namespace

// An instantiated step sequence, reused while everything it captured is unchanged.
struct BatchGraph {
  int mode;
  int64_t nsteps;
  int parity, blocks_per_sm, tile, extra, fallback;
  long long limit;
  double eps;
  cudaGraphExec_t exec;
};

struct elbm_batch_ctx {
  int ndom = 0;
  std::vector<int> edges;
  std::vector<long long> offs;
  std::vector<std::vector<double>> T;  // per-domain T (host copy, FP64)
  long long total = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;   // created when the caller passed the default stream
  int in_graph = -1;
  int tile = 256, blocks_per_sm = 0, nsm = 0;
  int ntiles = 0;
  DomainInfo* d_dom = nullptr;
  int* d_tile_dom = nullptr;
  int* d_tile_first = nullptr;
  float* buf[2] = {nullptr, nullptr};
  unsigned long long* d_fb = nullptr;
  unsigned* d_bar = nullptr;  // count, generation
  int* d_err = nullptr;
  int parity = 0;             // 0: state in buf[0]
  long long limit = 2000000000ll;
  int extra = 0;
  double eps = 0.0;
  int fallback = 1;
  bool initialized = false;
  int64_t step = 0;
  std::vector<BatchGraph> graphs;   // most recently used last
  std::string err;
};

namespace {

void drop_graphs(elbm_batch_ctx* h) {
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

cudaGraphExec_t find_graph(elbm_batch_ctx* h, int mode, int64_t nsteps) {
  for (size_t i = 0; i < h->graphs.size(); ++i) {
    const BatchGraph& g = h->graphs[i];
    if (g.mode == mode && g.nsteps == nsteps && g.parity == h->parity && g.blocks_per_sm == h->blocks_per_sm &&
        g.tile == h->tile && g.extra == h->extra && g.fallback == h->fallback && g.limit == h->limit &&
        g.eps == h->eps) {
      BatchGraph hit = g;
      h->graphs.erase(h->graphs.begin() + i);
      h->graphs.push_back(hit);
      return hit.exec;
    }
  }
  return nullptr;
}

void keep_graph(elbm_batch_ctx* h, int mode, int64_t nsteps, cudaGraphExec_t exec) {
  constexpr size_t kMax = 8;
  if (h->graphs.size() >= kMax) {
    cudaGraphExecDestroy(h->graphs.front().exec);
    h->graphs.erase(h->graphs.begin());
  }
  h->graphs.push_back(BatchGraph{mode, nsteps, h->parity, h->blocks_per_sm, h->tile, h->extra, h->fallback, h->limit,
                                 h->eps, exec});
}

elbm_status bfail(elbm_batch_ctx* h, elbm_status s, const std::string& m) {
  if (h) h->err = m;
  return s;
}
#define BCK(call, where)                                                                           \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return bfail(h, e_ == cudaErrorMemoryAllocation ? ELBM_ERR_OOM : ELBM_ERR_CUDA,              \
                   std::string(where) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

bool dptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

BatchArgs args_of(elbm_batch_ctx* h) {
  BatchArgs a;
  a.dom = h->d_dom;
  a.tile_dom = h->d_tile_dom;
  a.tile_first = h->d_tile_first;
  a.ntiles = h->ntiles;
  a.bufA = h->buf[0];
  a.bufB = h->buf[1];
  a.fb_count = h->d_fb;
  a.eps = (float)h->eps;
  a.fallback = h->fallback;
  return a;
}

elbm_status rebuild_tiles(elbm_batch_ctx* h) {
  // cached graphs hold the tile tables' addresses
  cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  std::vector<int> td, tf;
  for (int d = 0; d < h->ndom; ++d) {
    const int N = h->edges[d] * h->edges[d] * h->edges[d];
    for (int f = 0; f < N; f += h->tile) {
      td.push_back(d);
      tf.push_back(f);
    }
  }
  h->ntiles = (int)td.size();
  cudaFree(h->d_tile_dom);
  cudaFree(h->d_tile_first);
  h->d_tile_dom = h->d_tile_first = nullptr;
  BCK(cudaMalloc((void**)&h->d_tile_dom, td.size() * sizeof(int)), "cudaMalloc");
  BCK(cudaMalloc((void**)&h->d_tile_first, tf.size() * sizeof(int)), "cudaMalloc");
  BCK(cudaMemcpy(h->d_tile_dom, td.data(), td.size() * sizeof(int), cudaMemcpyHostToDevice), "memcpy");
  BCK(cudaMemcpy(h->d_tile_first, tf.data(), tf.size() * sizeof(int), cudaMemcpyHostToDevice), "memcpy");
  return ELBM_OK;
}

// one launch of the persistent kernel (not captured)
cudaError_t launch_persistent(elbm_batch_ctx* h, int nsteps, int grid) {
  BatchArgs a = args_of(h);
  int parity = h->parity;
  unsigned expected = (unsigned)(grid + h->extra);
  long long limit = h->limit;
  void* params[] = {&a, &nsteps, &parity, &h->d_bar, &expected, &limit, &h->d_err};
  cudaError_t e = cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((const void*)k_batch_persistent, dim3(grid), dim3(h->tile), params, 0, h->stream);
}

}  // namespace

extern "C" {

elbm_status elbm_batch_create(int32_t ndom, const int32_t* edges, const double* D6, void* cuda_stream,
                              elbm_batch_handle* out) {
  if (!out || !edges || !D6 || ndom < 1) return ELBM_ERR_ARG;
  *out = nullptr;
  elbm_batch_ctx* h = new elbm_batch_ctx();
  h->ndom = ndom;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  if (h->stream == nullptr) {
    // graph capture is not possible on the legacy default stream; this stream still
    // synchronises with it
    if (cudaStreamCreate(&h->own_stream) != cudaSuccess) {
      delete h;
      return ELBM_ERR_CUDA;
    }
    h->stream = h->own_stream;
  }
  std::vector<DomainInfo> info(ndom);
  long long off = 0;
  for (int d = 0; d < ndom; ++d) {
    const int n = edges[d];
    if (n < 1 || n > 256) {
      delete h;
      return ELBM_ERR_ARG;
    }
    double T[6];
    if (elbm_relaxation_complement(D6 + 6 * d, T) != ELBM_OK) {
      delete h;
      return ELBM_ERR_NOT_SPD;
    }
    h->edges.push_back(n);
    h->offs.push_back(off);
    h->T.emplace_back(T, T + 6);
    info[d].off = off;
    info[d].n = n;
    info[d].inv_n = 1.0f / (float)n;
    for (int q = 0; q < 6; ++q) info[d].T[q] = (float)T[q];
    off += (long long)n * n * n;
  }
  h->total = off;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaMalloc((void**)&h->d_dom, ndom * sizeof(DomainInfo));
  if (e == cudaSuccess) e = cudaMemcpy(h->d_dom, info.data(), ndom * sizeof(DomainInfo), cudaMemcpyHostToDevice);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc((void**)&h->buf[b], 27ull * off * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_fb, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_bar, 2 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->d_fb, 0, sizeof(unsigned long long));
  if (e != cudaSuccess) {
    elbm_status s = e == cudaErrorMemoryAllocation ? ELBM_ERR_OOM : ELBM_ERR_CUDA;
    elbm_batch_destroy(h);
    return s;
  }
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_batch_persistent, 256, 0);
  h->blocks_per_sm = std::max(1, bps);
  if (rebuild_tiles(h) != ELBM_OK) {
    elbm_batch_destroy(h);
    return ELBM_ERR_CUDA;
  }
  *out = h;
  return ELBM_OK;
}

void elbm_batch_destroy(elbm_batch_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  cudaFree(h->d_dom);
  cudaFree(h->d_tile_dom);
  cudaFree(h->d_tile_first);
  cudaFree(h->buf[0]);
  cudaFree(h->buf[1]);
  cudaFree(h->d_fb);
  cudaFree(h->d_bar);
  cudaFree(h->d_err);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
}

const char* elbm_batch_last_error(elbm_batch_handle h) { return h ? h->err.c_str() : "null handle"; }

elbm_status elbm_batch_info(elbm_batch_handle h, int64_t* total_nodes, int32_t* tile, int32_t* blocks_per_sm,
                            int32_t* persistent_in_graph) {
  if (!h) return ELBM_ERR_ARG;
  if (total_nodes) *total_nodes = h->total;
  if (tile) *tile = h->tile;
  if (blocks_per_sm) *blocks_per_sm = h->blocks_per_sm;
  if (persistent_in_graph) *persistent_in_graph = h->in_graph;
  return ELBM_OK;
}

elbm_status elbm_batch_set_params(elbm_batch_handle h, double eps, int32_t fallback) {
  if (!h || !std::isfinite(eps)) return bfail(h, ELBM_ERR_ARG, "bad params");
  h->eps = eps;
  h->fallback = fallback != 0;
  return ELBM_OK;
}

elbm_status elbm_batch_set_wait_limit(elbm_batch_handle h, int64_t cycles, int32_t extra_arrivals) {
  if (!h || cycles < 1 || extra_arrivals < 0) return bfail(h, ELBM_ERR_ARG, "bad wait limit");
  h->limit = cycles;
  h->extra = extra_arrivals;
  return ELBM_OK;
}

elbm_status elbm_batch_init_equilibrium(elbm_batch_handle h, const float* phi0) {
  if (!h || !phi0) return bfail(h, ELBM_ERR_ARG, "null argument");
  const float* dev = phi0;
  float* tmp = nullptr;
  if (!dptr(phi0)) {
    BCK(cudaMallocAsync((void**)&tmp, h->total * sizeof(float), h->stream), "cudaMallocAsync");
    BCK(cudaMemcpyAsync(tmp, phi0, h->total * sizeof(float), cudaMemcpyHostToDevice, h->stream), "memcpy");
    dev = tmp;
  }
  const int grid = std::min(h->ntiles, 65535 * 8);
  k_batch_write<<<grid, h->tile, 0, h->stream>>>(h->d_dom, h->d_tile_dom, h->d_tile_first, h->ntiles, dev, h->buf[0]);
  BCK(cudaGetLastError(), "init kernel");
  if (tmp) BCK(cudaFreeAsync(tmp, h->stream), "free");
  BCK(cudaMemsetAsync(h->d_fb, 0, sizeof(unsigned long long), h->stream), "memset");
  BCK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream), "memset");
  h->parity = 0;
  h->step = 0;
  h->initialized = true;
  return ELBM_OK;
}

elbm_status elbm_batch_step(elbm_batch_handle h, int64_t nsteps, int32_t mode) {
  if (!h || nsteps < 0 || mode < 0 || mode > 2) return bfail(h, ELBM_ERR_ARG, "bad argument");
  if (!h->initialized) return bfail(h, ELBM_ERR_STATE, "not initialised");
  if (nsteps == 0) return ELBM_OK;
  if (mode == 2) {
    // reference path: one plain single-lattice launch per domain per step
    for (int64_t s = 0; s < nsteps; ++s) {
      const float* in = h->buf[h->parity];
      float* outb = h->buf[1 - h->parity];
      for (int d = 0; d < h->ndom; ++d) {
        const int n = h->edges[d];
        PopConsts<float> kf{};
        for (int i = 0; i < Q; ++i) kf.E[i] = (float)w_of(i);
        kf.eps = (float)h->eps;
        const auto& T = h->T[d];
        kf.T = Sym6<float>{(float)T[0], (float)T[1], (float)T[2], (float)T[3], (float)T[4], (float)T[5]};
        StepLaunch L{};
        L.prec = 1;
        L.vel = 0;
        L.nx = L.ny = L.nz = n;
        L.N = (size_t)n * n * n;
        L.dirichlet = 0;
        L.fallback = h->fallback;
        L.pin = in + 27ll * h->offs[d];
        L.pout = outb + 27ll * h->offs[d];
        L.counters = h->d_fb;
        L.kf = &kf;
        BCK(launch_step(L, h->stream), "per-domain step");
      }
      h->parity ^= 1;
    }
    h->step += nsteps;
    return ELBM_OK;
  }
  // a step sequence captured before with the same shape, state parity and parameters is
  // relaunched as it is: capture and instantiation stay out of repeated calls
  if (cudaGraphExec_t cached = find_graph(h, mode, nsteps)) {
    BCK(cudaGraphLaunch(cached, h->stream), "graph launch");
    if (nsteps % 2) h->parity ^= 1;
    h->step += nsteps;
    return ELBM_OK;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  BCK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = cudaSuccess;
  if (mode == 0) {
    e = launch_persistent(h, (int)nsteps, h->blocks_per_sm * h->nsm);
  } else {
    BatchArgs a = args_of(h);
    int parity = h->parity;
    const int grid = h->blocks_per_sm * h->nsm * 4;
    for (int64_t s = 0; s < nsteps && e == cudaSuccess; ++s) {
      k_batch_step<<<grid, h->tile, 0, h->stream>>>(a, parity);
      e = cudaGetLastError();
      parity ^= 1;
    }
  }
  cudaError_t ec = cudaStreamEndCapture(h->stream, &graph);
  if (e != cudaSuccess || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (mode == 0) {
      // capture of the cooperative launch refused: launch it directly
      h->in_graph = 0;
      BCK(launch_persistent(h, (int)nsteps, h->blocks_per_sm * h->nsm), "persistent launch");
      if (nsteps % 2) h->parity ^= 1;
      h->step += nsteps;
      return ELBM_OK;
    }
    return bfail(h, ELBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : ec));
  }
  if (mode == 0) h->in_graph = 1;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, h->stream);
  if (e != cudaSuccess) {
    if (exec) cudaGraphExecDestroy(exec);
    return bfail(h, ELBM_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  }
  keep_graph(h, mode, nsteps, exec);
  if (nsteps % 2) h->parity ^= 1;
  h->step += nsteps;
  return ELBM_OK;
}

elbm_status elbm_batch_synchronize(elbm_batch_handle h) {
  if (!h) return ELBM_ERR_ARG;
  BCK(cudaStreamSynchronize(h->stream), "sync");
  int err = 0;
  BCK(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost), "memcpy");
  if (err) return bfail(h, ELBM_ERR_TIMEOUT, "a grid-barrier wait ran out; the state is incomplete");
  return ELBM_OK;
}

elbm_status elbm_batch_autotune(elbm_batch_handle h, int32_t steps_per_trial, int32_t* tile_out,
                                int32_t* blocks_per_sm_out) {
  if (!h || steps_per_trial < 1) return bfail(h, ELBM_ERR_ARG, "bad argument");
  if (!h->initialized) return bfail(h, ELBM_ERR_STATE, "not initialised");
  // candidates: threads per block (tile) 128 or 256; resident blocks per SM 1..occupancy
  int best_b = h->blocks_per_sm, best_t = h->tile;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int t : {128, 256})
  for (int b = 1;; ++b) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_persistent, t, 0);
    if (b > std::max(1, occ)) break;
    if (h->tile != t) {
      h->tile = t;
      if (rebuild_tiles(h) != ELBM_OK) break;
    }
    h->blocks_per_sm = b;
    cudaEventRecord(e0, h->stream);
    elbm_status s = elbm_batch_step(h, steps_per_trial, 0);
    cudaEventRecord(e1, h->stream);
    if (s != ELBM_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return s;
    }
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best_b = b;
      best_t = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->blocks_per_sm = best_b;
  if (h->tile != best_t) {
    h->tile = best_t;
    elbm_status s = rebuild_tiles(h);
    if (s != ELBM_OK) return s;
  }
  if (tile_out) *tile_out = h->tile;
  if (blocks_per_sm_out) *blocks_per_sm_out = best_b;
  return elbm_batch_synchronize(h);
}

elbm_status elbm_batch_read_phi(elbm_batch_handle h, float* phi) {
  if (!h || !phi) return bfail(h, ELBM_ERR_ARG, "null argument");
  if (!h->initialized) return bfail(h, ELBM_ERR_STATE, "not initialised");
  const bool host = !dptr(phi);
  float* dst = phi;
  if (host) BCK(cudaMallocAsync((void**)&dst, h->total * sizeof(float), h->stream), "cudaMallocAsync");
  const int grid = std::min(h->ntiles, 65535 * 8);
  k_batch_read<<<grid, h->tile, 0, h->stream>>>(h->d_dom, h->d_tile_dom, h->d_tile_first, h->ntiles,
                                               h->buf[h->parity], dst, nullptr, -1);
  BCK(cudaGetLastError(), "read kernel");
  if (host) {
    BCK(cudaMemcpyAsync(phi, dst, h->total * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "memcpy");
    BCK(cudaFreeAsync(dst, h->stream), "free");
    BCK(cudaStreamSynchronize(h->stream), "sync");
  }
  return ELBM_OK;
}

elbm_status elbm_batch_read_populations(elbm_batch_handle h, int32_t domain, float* out) {
  if (!h || !out || domain < 0 || domain >= h->ndom) return bfail(h, ELBM_ERR_ARG, "bad argument");
  if (!h->initialized) return bfail(h, ELBM_ERR_STATE, "not initialised");
  const long long N = (long long)h->edges[domain] * h->edges[domain] * h->edges[domain];
  const bool host = !dptr(out);
  float* dst = out;
  if (host) BCK(cudaMallocAsync((void**)&dst, 27 * N * sizeof(float), h->stream), "cudaMallocAsync");
  const int grid = std::min(h->ntiles, 65535 * 8);
  k_batch_read<<<grid, h->tile, 0, h->stream>>>(h->d_dom, h->d_tile_dom, h->d_tile_first, h->ntiles,
                                               h->buf[h->parity], nullptr, dst, domain);
  BCK(cudaGetLastError(), "read kernel");
  if (host) {
    BCK(cudaMemcpyAsync(out, dst, 27 * N * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "memcpy");
    BCK(cudaFreeAsync(dst, h->stream), "free");
    BCK(cudaStreamSynchronize(h->stream), "sync");
  }
  return ELBM_OK;
}

elbm_status elbm_batch_fallback_count(elbm_batch_handle h, int64_t* n) {
  if (!h || !n) return bfail(h, ELBM_ERR_ARG, "null argument");
  unsigned long long v = 0;
  BCK(cudaMemcpyAsync(&v, h->d_fb, sizeof(v), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  BCK(cudaStreamSynchronize(h->stream), "sync");
  *n = (int64_t)v;
  return ELBM_OK;
}

}  // extern "C"
