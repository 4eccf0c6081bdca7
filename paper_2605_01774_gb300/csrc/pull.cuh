// Pull streaming (Eq. method-lbe read backwards): node x gathers A_i(x - c_i)
// from the post-collision buffer.  Periodic wrap in every axis, or halfway
// anti-bounce-back x faces: at x = 0 the populations entering with c_x = +1, and
// at x = Nx-1 those entering with c_x = -1, are
//     g_i(x_b) = -A_opp(i)(x_b) + 2 W_i phi_w        (wall velocity 0).
#pragma once
#include "collide.cuh"
#include "storage.cuh"

namespace elbm {

template <typename Elem>
struct Field {
  const Elem* pops;     // [27][N] storage elements
  const float* scale;   // [N] deviation scale (deviation formats), else unused
};

struct Grid {
  int nx, ny, nz;
  size_t N;
  int dirichlet;
};

template <typename Elem, typename R>
__device__ __forceinline__ void pull_node(R (&g)[Q], const Field<Elem>& f, const Grid& G, int x, int y, int z,
                                          const PopConsts<R>& k) {
  using ST = Storage<Elem>;
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const int nxy = nx * ny;
  // source coordinate for velocity component c in {-1, 0, +1} is coordinate - c
  const int xs[3] = {x + 1 == nx ? 0 : x + 1, x, x == 0 ? nx - 1 : x - 1};
  const int ys[3] = {(y + 1 == ny ? 0 : y + 1) * nx, y * nx, (y == 0 ? ny - 1 : y - 1) * nx};
  const int zs[3] = {(z + 1 == nz ? 0 : z + 1) * nxy, z * nxy, (z == 0 ? nz - 1 : z - 1) * nxy};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int src = xs[cx_of(i) + 1] + ys[cy_of(i) + 1] + zs[cz_of(i) + 1];
    g[i] = ST::load(f.pops, f.scale, G.N, i, src, k.E[i]);
  }
  if (G.dirichlet && (x == 0 || x == nx - 1)) {
    const int n = x + ys[1] + zs[1];
    if (x == 0) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        if (cx_of(i) == 1)
          g[i] = R(2.0 * w_of(i)) * k.phi_lo - ST::load(f.pops, f.scale, G.N, opp_of(i), n, k.E[opp_of(i)]);
    }
    if (x == nx - 1) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        if (cx_of(i) == -1)
          g[i] = R(2.0 * w_of(i)) * k.phi_hi - ST::load(f.pops, f.scale, G.N, opp_of(i), n, k.E[opp_of(i)]);
    }
  }
}

// Per-node T = 2I - S: stored in the arithmetic type R ([6][N]); null = uniform.
template <typename R>
__device__ __forceinline__ Sym6<R> load_T(const R* __restrict__ T6, size_t N, int n, const Sym6<R>& uni) {
  if (T6 == nullptr) return uni;
  Sym6<R> t;
  t.xx = __ldg(T6 + n);
  t.xy = __ldg(T6 + N + n);
  t.xz = __ldg(T6 + 2 * N + n);
  t.yy = __ldg(T6 + 3 * N + n);
  t.yz = __ldg(T6 + 4 * N + n);
  t.zz = __ldg(T6 + 5 * N + n);
  return t;
}

}  // namespace elbm
