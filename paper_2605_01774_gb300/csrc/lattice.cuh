// D3Q27 velocity set and weights as compile-time functions (Section 2.1).
// Population i has velocity (cx, cy, cz) with i = 9 (cx+1) + 3 (cy+1) + (cz+1);
// loops over i are fully unrolled so every c_i and W_i folds to a constant.
#pragma once
#include <cstdint>

namespace elbm {

constexpr int Q = 27;

__host__ __device__ constexpr int cx_of(int i) { return i / 9 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int opp_of(int i) { return 26 - i; }
__host__ __device__ constexpr int nnz_of(int i) {
  return (cx_of(i) != 0) + (cy_of(i) != 0) + (cz_of(i) != 0);
}
// Exponent e_i = 2 + 2 m (m = number of nonzero components of c_i) of the scaling of the
// stored deviations: W_i 2^e_i = 32/27 for every i.
__host__ __device__ constexpr int qexp_of(int i) { return 2 + 2 * nnz_of(i); }
// W_i = (2/3)^(3-m) (1/6)^m: 8/27, 2/27, 1/54, 1/216 for m = 0..3
__host__ __device__ constexpr double w_of(int i) {
  return nnz_of(i) == 0 ? 8.0 / 27.0 : nnz_of(i) == 1 ? 2.0 / 27.0 : nnz_of(i) == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
}

// Symmetric 3x3 stored as (xx, xy, xz, yy, yz, zz).
template <typename R>
struct Sym6 {
  R xx, xy, xz, yy, yz, zz;
};

template <typename R>
__host__ __device__ __forceinline__ void sym_mul(const Sym6<R>& M, R vx, R vy, R vz, R& ox, R& oy, R& oz) {
  ox = M.xx * vx + M.xy * vy + M.xz * vz;
  oy = M.xy * vx + M.yy * vy + M.yz * vz;
  oz = M.xz * vx + M.yz * vy + M.zz * vz;
}

}  // namespace elbm
