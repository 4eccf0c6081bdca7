// State transfer, read-outs, conservation reductions and the tensor pre-pass.
#include <cfloat>

#include "internal.h"
#include "pull.cuh"

namespace elbm {

namespace {

dim3 block2d(int nx) {
  int bx = nx >= 256 ? 256 : ((nx + 31) / 32) * 32;
  return dim3(bx, 256 / bx, 1);
}
dim3 grid2d(dim3 b, int nx, int ny, int nz) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y, nz); }

template <typename T>
__device__ __forceinline__ double ld_in(const void* p, size_t idx) {
  return (double)static_cast<const T*>(p)[idx];
}

// ---------------------------------------------------------------- write state
// Stored layout is post-collision: the next step pulls A_i(y) into node y + c_i
// and adds R E_i there.  To make the next step see the pre-collision state G
// (which already holds the trailing half source), store
//   A_i(y) = G_i(y + c_i) - (1/2) R(y + c_i) E_i         if y + c_i is a node,
//   A_i(y) = 2 W_i phi_w - (G_opp(i)(y) - (1/2) R(y) E_opp(i))   otherwise
// (anti-bounce-back inverted: the stored outgoing population of a wall node only
// feeds the entering opposite one).
template <typename Elem, typename Tin, int FROM_PHI>
__global__ void __launch_bounds__(256)
k_write(Elem* __restrict__ pops, float* __restrict__ scale, Grid G, const void* __restrict__ in,
        const float* __restrict__ src, const float* __restrict__ u3,
        const PopConsts<typename Storage<Elem>::real> k) {
  using R = typename Storage<Elem>::real;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= G.nx || y >= G.ny) return;
  const int n = x + G.nx * (y + G.ny * z);
  R a[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int dx = x + cx_of(i), dy = y + cy_of(i), dz = z + cz_of(i);
    const bool through_hi = dx >= G.nx;  // leaves through x = Nx - 1/2 (else through x = -1/2)
    dy = dy < 0 ? G.ny - 1 : (dy >= G.ny ? 0 : dy);
    dz = dz < 0 ? G.nz - 1 : (dz >= G.nz ? 0 : dz);
    const bool outside = G.dirichlet && (dx < 0 || dx >= G.nx);
    dx = dx < 0 ? G.nx - 1 : (dx >= G.nx ? 0 : dx);
    const int d = dx + G.nx * (dy + G.ny * dz);
    if (!outside) {
      R Ei = k.E[i];
      if (FROM_PHI && u3 != nullptr) {   // equilibrium at the velocity of node d
        const R ux = u3[d], uy = u3[G.N + d], uz = u3[2 * G.N + d];
        const R cu = R(cx_of(i)) * ux + R(cy_of(i)) * uy + R(cz_of(i)) * uz;
        Ei = R(w_of(i)) * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * (ux * ux + uy * uy + uz * uz));
      }
      R v = FROM_PHI ? R(ld_in<Tin>(in, d)) * Ei : R(ld_in<Tin>(in, (size_t)i * G.N + d));
      if (src != nullptr) v -= k.src_half * R(src[d]) * k.E[i];
      a[i] = v;
    } else {
      const int o = opp_of(i);
      R Eo = k.E[o];
      if (FROM_PHI && u3 != nullptr) {
        const R ux = u3[n], uy = u3[G.N + n], uz = u3[2 * G.N + n];
        const R cu = R(cx_of(o)) * ux + R(cy_of(o)) * uy + R(cz_of(o)) * uz;
        Eo = R(w_of(o)) * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * (ux * ux + uy * uy + uz * uz));
      }
      R v = FROM_PHI ? R(ld_in<Tin>(in, n)) * Eo : R(ld_in<Tin>(in, (size_t)o * G.N + n));
      if (src != nullptr) v -= k.src_half * R(src[n]) * k.E[o];
      const R phw = through_hi ? k.phi_hi : k.phi_lo;
      a[i] = R(2.0 * w_of(i)) * phw - v;
    }
  }
  Storage<Elem>::store(pops, scale, G.N, n, a, k.Ek, R(NAN));
}

// ----------------------------------------------------------------- read state
template <typename Elem, typename Tout, int WHAT>
__global__ void __launch_bounds__(256)
k_read(Field<Elem> f, Grid G, Tout* __restrict__ out, Tout* __restrict__ qout,
       const typename Storage<Elem>::real* __restrict__ T6,
       const float* __restrict__ src, const float* __restrict__ u3,
       const PopConsts<typename Storage<Elem>::real> k) {
  using R = typename Storage<Elem>::real;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= G.nx || y >= G.ny) return;
  const int n = x + G.nx * (y + G.ny * z);
  R g[Q];
  pull_node<Elem, R>(g, f, G, x, y, z, k);
  if (src != nullptr) {
    const R r = k.src_half * R(src[n]);
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] += r * k.E[i];
  }
  if (WHAT == 0) {
#pragma unroll
    for (int i = 0; i < Q; ++i) out[(size_t)i * G.N + n] = Tout(g[i]);
  } else {
    R phi, mx, my, mz;
    moments(g, phi, mx, my, mz);
    out[n] = Tout(phi);
    if (qout != nullptr) {
      // q = j - S j / 2 = T j / 2 with T = 2I - S (Eq. app-cube-lb-flux)
      R ux = k.ux, uy = k.uy, uz = k.uz;
      if (u3 != nullptr) {
        ux = u3[n];
        uy = u3[G.N + n];
        uz = u3[2 * G.N + n];
      }
      const R jx = mx - phi * ux, jy = my - phi * uy, jz = mz - phi * uz;
      const Sym6<R> T = load_T<R>(T6, G.N, n, k.T);
      R tx, ty, tz;
      sym_mul(T, jx, jy, jz, tx, ty, tz);
      qout[n] = Tout(R(0.5) * tx);
      qout[G.N + n] = Tout(R(0.5) * ty);
      qout[2 * G.N + n] = Tout(R(0.5) * tz);
    }
  }
}

// ----------------------------------------------------------------- reductions
// Per block: sum phi, sum g ln(g/W) over g > 0, min g, count of non-finite g;
// one partial per block, then a single block adds the partials in index order.
template <typename Elem>
__global__ void __launch_bounds__(256)
k_reduce_partials(Field<Elem> f, Grid G, const float* __restrict__ src, double* __restrict__ part,
                  const PopConsts<typename Storage<Elem>::real> k) {
  using R = typename Storage<Elem>::real;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  double m = 0.0, h = 0.0, gmin = DBL_MAX, bad = 0.0;
  if (x < G.nx && y < G.ny) {
    const int n = x + G.nx * (y + G.ny * z);
    R g[Q];
    pull_node<Elem, R>(g, f, G, x, y, z, k);
    const double r = src != nullptr ? (double)k.src_half * (double)src[n] : 0.0;
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
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
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
  if (tid == 0) {
    const int nw = (blockDim.x * blockDim.y + 31) / 32;
    double a = 0, b = 0, c = DBL_MAX, d = 0;
    for (int w = 0; w < nw; ++w) {
      a += sm[0][w];
      b += sm[1][w];
      c = fmin(c, sm[2][w]);
      d += sm[3][w];
    }
    const size_t blk = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    part[4 * blk + 0] = a;
    part[4 * blk + 1] = b;
    part[4 * blk + 2] = c;
    part[4 * blk + 3] = d;
  }
}

__global__ void __launch_bounds__(1024) k_reduce_final(const double* __restrict__ part, size_t nblk,
                                                       double* __restrict__ out4) {
  __shared__ double sm[4][1024];
  double a = 0, b = 0, c = DBL_MAX, d = 0;
  for (size_t i = threadIdx.x; i < nblk; i += blockDim.x) {
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

// ---------------------------------------------------------------- tensor pre-pass
// T = 2I - S = 12 D (I + 6 D)^-1 per node, in FP64 (Eq. method-s-from-d with
// cs2 = 1/3, dt = 1), from Cartesian D or from (ln d_k, ZYZ angles).
__device__ void sym3_inverse(const double m[6], double inv[6], double& det) {
  const double a = m[0], b = m[1], c = m[2], d = m[3], e = m[4], f = m[5];
  const double A = d * f - e * e, B = c * e - b * f, C = b * e - c * d;
  det = a * A + b * B + c * C;
  const double id = 1.0 / det;
  inv[0] = A * id;
  inv[1] = B * id;
  inv[2] = C * id;
  inv[3] = (a * f - c * c) * id;
  inv[4] = (b * c - a * e) * id;
  inv[5] = (a * d - b * b) * id;
}

template <typename TT>
__global__ void k_tensor(const float* __restrict__ in, int is_params, TT* __restrict__ T6, size_t N,
                         unsigned long long* bad) {
  const size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  double t6[6];
  if (is_params) {
    double t[3];
    for (int k = 0; k < 3; ++k) {
      const double dk = exp((double)in[k * N + n]);
      t[k] = 12.0 * dk / (1.0 + 6.0 * dk);
    }
    double sa, ca, sb, cb, sc, cc;
    sincos((double)in[3 * N + n], &sa, &ca);
    sincos((double)in[4 * N + n], &sb, &cb);
    sincos((double)in[5 * N + n], &sc, &cc);
    // R = Rz(a) Ry(b) Rz(c)
    const double R[3][3] = {{ca * cb * cc - sa * sc, -ca * cb * sc - sa * cc, ca * sb},
                            {sa * cb * cc + ca * sc, -sa * cb * sc + ca * cc, sa * sb},
                            {-sb * cc, sb * sc, cb}};
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6; ++q) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += R[ia[q]][k] * t[k] * R[ib[q]][k];
      t6[q] = s;
    }
    if (!(isfinite(t[0]) && isfinite(t[1]) && isfinite(t[2]))) atomicAdd(bad, 1ull);
  } else {
    double D[6];
    for (int q = 0; q < 6; ++q) D[q] = in[q * N + n];
    // Sylvester criterion for SPD
    const double m1 = D[0], m2 = D[0] * D[3] - D[1] * D[1];
    const double det = D[0] * (D[3] * D[5] - D[4] * D[4]) - D[1] * (D[1] * D[5] - D[4] * D[2]) +
                       D[2] * (D[1] * D[4] - D[3] * D[2]);
    if (!(m1 > 0.0 && m2 > 0.0 && det > 0.0)) atomicAdd(bad, 1ull);
    double M[6] = {1.0 + 6.0 * D[0], 6.0 * D[1], 6.0 * D[2], 1.0 + 6.0 * D[3], 6.0 * D[4], 1.0 + 6.0 * D[5]};
    double Mi[6], dm;
    sym3_inverse(M, Mi, dm);
    // 12 D Mi (D and Mi commute, product symmetric)
    const double Dm[3][3] = {{D[0], D[1], D[2]}, {D[1], D[3], D[4]}, {D[2], D[4], D[5]}};
    const double Im[3][3] = {{Mi[0], Mi[1], Mi[2]}, {Mi[1], Mi[3], Mi[4]}, {Mi[2], Mi[4], Mi[5]}};
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6; ++q) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += Dm[ia[q]][k] * Im[k][ib[q]];
      t6[q] = 12.0 * s;
    }
  }
  for (int q = 0; q < 6; ++q) T6[q * N + n] = (TT)t6[q];
}

template <typename Elem>
Field<Elem> field_of(const StateIO& S) {
  return Field<Elem>{static_cast<const Elem*>(S.pops), S.scale};
}

template <typename Elem>
const PopConsts<typename Storage<Elem>::real>& consts_of(const StateIO& S) {
  using R = typename Storage<Elem>::real;
  return *reinterpret_cast<const PopConsts<R>*>(std::is_same<R, double>::value ? (const void*)S.kd : (const void*)S.kf);
}

template <typename Elem>
cudaError_t write_t(const StateIO& S, const void* in, int in_f32, int from_phi, cudaStream_t s) {
  Grid G{S.nx, S.ny, S.nz, S.N, S.dirichlet};
  dim3 b = block2d(S.nx), g = grid2d(b, S.nx, S.ny, S.nz);
  Elem* p = static_cast<Elem*>(S.pops);
  const auto& k = consts_of<Elem>(S);
  if (in_f32) {
    if (from_phi) k_write<Elem, float, 1><<<g, b, 0, s>>>(p, S.scale, G, in, S.src, S.u3, k);
    else k_write<Elem, float, 0><<<g, b, 0, s>>>(p, S.scale, G, in, S.src, S.u3, k);
  } else {
    if (from_phi) k_write<Elem, double, 1><<<g, b, 0, s>>>(p, S.scale, G, in, S.src, S.u3, k);
    else k_write<Elem, double, 0><<<g, b, 0, s>>>(p, S.scale, G, in, S.src, S.u3, k);
  }
  return cudaGetLastError();
}

template <typename Elem>
cudaError_t read_t(const StateIO& S, void* out, void* q, int out_f32, int what, cudaStream_t s) {
  Grid G{S.nx, S.ny, S.nz, S.N, S.dirichlet};
  dim3 b = block2d(S.nx), g = grid2d(b, S.nx, S.ny, S.nz);
  using R = typename Storage<Elem>::real;
  const auto& k = consts_of<Elem>(S);
  Field<Elem> f = field_of<Elem>(S);
  const R* T6 = static_cast<const R*>(S.T6);
  if (out_f32) {
    if (what == 0) k_read<Elem, float, 0><<<g, b, 0, s>>>(f, G, (float*)out, (float*)q, T6, S.src, S.u3, k);
    else k_read<Elem, float, 1><<<g, b, 0, s>>>(f, G, (float*)out, (float*)q, T6, S.src, S.u3, k);
  } else {
    if (what == 0) k_read<Elem, double, 0><<<g, b, 0, s>>>(f, G, (double*)out, (double*)q, T6, S.src, S.u3, k);
    else k_read<Elem, double, 1><<<g, b, 0, s>>>(f, G, (double*)out, (double*)q, T6, S.src, S.u3, k);
  }
  return cudaGetLastError();
}

template <typename Elem>
cudaError_t reduce_t(const StateIO& S, double* scratch, double* out4, cudaStream_t s) {
  Grid G{S.nx, S.ny, S.nz, S.N, S.dirichlet};
  dim3 b = block2d(S.nx), g = grid2d(b, S.nx, S.ny, S.nz);
  k_reduce_partials<Elem><<<g, b, 0, s>>>(field_of<Elem>(S), G, S.src, scratch, consts_of<Elem>(S));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_final<<<1, 1024, 0, s>>>(scratch, (size_t)g.x * g.y * g.z, out4);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_write_state(const StateIO& S, const void* in, int in_f32, int from_phi, cudaStream_t s) {
  switch (S.prec) {
    case 0: return write_t<double>(S, in, in_f32, from_phi, s);
    case 1: return write_t<float>(S, in, in_f32, from_phi, s);
    case 2: return write_t<__half>(S, in, in_f32, from_phi, s);
    case 3: return write_t<__nv_bfloat16>(S, in, in_f32, from_phi, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_read_state(const StateIO& S, void* out, void* q, int out_f32, int what, cudaStream_t s) {
  switch (S.prec) {
    case 0: return read_t<double>(S, out, q, out_f32, what, s);
    case 1: return read_t<float>(S, out, q, out_f32, what, s);
    case 2: return read_t<__half>(S, out, q, out_f32, what, s);
    case 3: return read_t<__nv_bfloat16>(S, out, q, out_f32, what, s);
  }
  return cudaErrorInvalidValue;
}

size_t reduce_blocks(const StateIO& S) {
  dim3 b = block2d(S.nx), g = grid2d(b, S.nx, S.ny, S.nz);
  return (size_t)g.x * g.y * g.z;
}

cudaError_t launch_reduce(const StateIO& S, double* scratch, double* out4, cudaStream_t s) {
  switch (S.prec) {
    case 0: return reduce_t<double>(S, scratch, out4, s);
    case 1: return reduce_t<float>(S, scratch, out4, s);
    case 2: return reduce_t<__half>(S, scratch, out4, s);
    case 3: return reduce_t<__nv_bfloat16>(S, scratch, out4, s);
  }
  return cudaErrorInvalidValue;
}

__global__ void k_velocity_check(const float* __restrict__ u3, size_t N, unsigned long long* bad) {
  const size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double ux = u3[n], uy = u3[N + n], uz = u3[2 * N + n];
  bool ok = isfinite(ux) && isfinite(uy) && isfinite(uz);
  const double uu = ux * ux + uy * uy + uz * uz;
  for (int i = 0; i < Q && ok; ++i) {
    const double cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
    ok = 1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu > 0.0;
  }
  if (!ok) atomicAdd(bad, 1ull);
}

cudaError_t launch_velocity_check(const float* u3, size_t N, unsigned long long* bad, cudaStream_t s) {
  const int b = 256;
  k_velocity_check<<<(unsigned)((N + b - 1) / b), b, 0, s>>>(u3, N, bad);
  return cudaGetLastError();
}

cudaError_t launch_tensor_prepass(const float* in, int is_params, void* T6, int t6_f64, size_t N,
                                  unsigned long long* bad, cudaStream_t s) {
  const int b = 256;
  const size_t g = (N + b - 1) / b;
  if (t6_f64) k_tensor<double><<<(unsigned)g, b, 0, s>>>(in, is_params, static_cast<double*>(T6), N, bad);
  else k_tensor<float><<<(unsigned)g, b, 0, s>>>(in, is_params, static_cast<float*>(T6), N, bad);
  return cudaGetLastError();
}

}  // namespace elbm
