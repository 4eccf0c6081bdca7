// Two-dimensional form of the fused collide-stream step on the D2Q9 tensor-product set
// (Section 2.1 defines the method on D2Q9 and D3Q27; Section 4.1 runs it on D2Q9 with
// tensor and velocity fields that vary in space), with its C ABI (include/elbm2d.h).
//
// One thread per node: pull the 9 populations from (x - cx, y - cy) with periodic wrap
// (coalesced along x; the rows y - 1, y, y + 1 of a plane are shared by neighbouring blocks
// through L1/L2), collide in registers, write the 9 results at the own node of the other
// buffer.  The collision is that of the three-dimensional kernel written for d = 2:
// phi = sum g, j = sum c g - phi u, a = (I - S) j = T j - j with T = 2I - S, and
//     g*_i = (1 + kappa) phi E_i - kappa g_i + 3 W_i c_i.(a + kappa j),
// kappa = lambda - 1 from Eqs. (method-lambda, method-correction) with the identically-zero
// terms removed, evaluated on phi-relative quantities, kappa = 0 where u = 0, where
// sum (dh/phi)^2 M <= theta^2 or where phi is not above 1e-30 (FP32) / 1e-300 (FP64); then
// the positivity fallback of Eq. (method-alpha).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>

#include "../../include/elbm2d.h"
#include "eqlog.cuh"

namespace {

constexpr int Q2 = 9;
__host__ __device__ constexpr int cx2(int i) { return i / 3 - 1; }
__host__ __device__ constexpr int cy2(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int nnz2(int i) { return (cx2(i) != 0) + (cy2(i) != 0); }
// W_i = (2/3)^(2 - m) (1/6)^m
__host__ __device__ constexpr double w2(int i) {
  return nnz2(i) == 0 ? 4.0 / 9.0 : (nnz2(i) == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
}

template <typename R>
struct Consts2 {
  R E[Q2];    // W_i P_i(u)
  R K3[Q2];   // 3 (1/P_i - 1)
  R L[Q2];    // ln P_i - 3 c_i.u + 1.5 u.u
  R M[Q2];    // 1 / (W_i P_i)
  R ux, uy;
  R theta2, eps;
  R txx, txy, tyy;   // uniform T = 2I - S
};

double poly2(int i, double ux, double uy) {
  const double cu = cx2(i) * ux + cy2(i) * uy;
  return 1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy);
}

template <typename R>
__device__ __forceinline__ void node_tables2(Consts2<R>& k, R ux, R uy) {
  const R uu = ux * ux + uy * uy;
#pragma unroll
  for (int i = 0; i < Q2; ++i) {
    const R cu = R(cx2(i)) * ux + R(cy2(i)) * uy;
    if constexpr (sizeof(R) == 4) {
      elbm::eq_tables_f32(fmaf(3.0f, cu, __fmul_rn(-1.5f, uu)), __fmul_rn(__fmul_rn(4.5f, cu), cu), float(w2(i)),
                          k.E[i], k.K3[i], k.L[i], k.M[i]);
    } else {
      const R P = R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu;
      const R rP = R(1) / P;   // one quotient serves K3 and M
      k.E[i] = R(w2(i)) * P;
      k.K3[i] = R(3) * (rP - R(1));
      k.L[i] = log(P) - R(3) * cu + R(1.5) * uu;
      k.M[i] = rP * R(1.0 / w2(i));
    }
  }
  k.ux = ux;
  k.uy = uy;
}

// VEL 0: u = 0 (kappa = 0); 1: uniform u (tables in k); 2: the node's own u (tables rebuilt).
// Returns true where the positivity fallback was taken.
template <typename R, int VEL>
__device__ __forceinline__ bool collide2(R (&g)[Q2], R txx, R txy, R tyy, const Consts2<R>& k, bool fallback) {
  R s[3], d[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    s[c] = g[3 * c] + g[3 * c + 1] + g[3 * c + 2];
    d[c] = g[3 * c + 2] - g[3 * c];
  }
  const R phi = s[0] + s[1] + s[2];
  R jx = s[2] - s[0], jy = d[0] + d[1] + d[2];
  if (VEL != 0) {
    jx -= phi * k.ux;
    jy -= phi * k.uy;
  }
  const R ax = txx * jx + txy * jy - jx, ay = txy * jx + tyy * jy - jy;   // (I - S) j
  R gs[Q2];
  if (VEL == 0) {
#pragma unroll
    for (int i = 0; i < Q2; ++i) gs[i] = phi * R(w2(i)) + R(3.0 * w2(i)) * (R(cx2(i)) * ax + R(cy2(i)) * ay);
  } else {
    R kappa = R(0);
    const R tiny = sizeof(R) == 4 ? R(1e-30) : R(1e-300);
    if (phi > tiny) {
      const R inv = sizeof(R) == 4 ? R(__fdividef(1.0f, float(phi))) : R(1) / phi;
      const R jxr = jx * inv, jyr = jy * inv, axr = ax * inv, ayr = ay * inv;
      R num = R(0), den = R(0);
#pragma unroll
      for (int i = 0; i < Q2; ++i) {
        R dh = g[i] * inv - k.E[i];
        dh = dh - R(3.0 * w2(i)) * (R(cx2(i)) * jxr + R(cy2(i)) * jyr);
        num += dh * (k.K3[i] * (R(cx2(i)) * axr + R(cy2(i)) * ayr) + k.L[i]);
        den += dh * (dh * k.M[i]);
      }
      if (den > k.theta2) kappa = sizeof(R) == 4 ? R(__fdividef(float(num), float(den))) : num / den;
    }
    const R psi = (R(1) + kappa) * phi;
    const R bx = ax + kappa * jx, by = ay + kappa * jy;
#pragma unroll
    for (int i = 0; i < Q2; ++i)
      gs[i] = psi * k.E[i] - kappa * g[i] + R(3.0 * w2(i)) * (R(cx2(i)) * bx + R(cy2(i)) * by);
  }
  bool took = false;
  if (fallback) {
    R mn = gs[0];
#pragma unroll
    for (int i = 1; i < Q2; ++i) mn = mn < gs[i] ? mn : gs[i];
    if (mn < k.eps) {
      took = true;
      R alpha = R(1);
#pragma unroll
      for (int i = 0; i < Q2; ++i) {
        if (gs[i] < k.eps && g[i] > gs[i]) {
          const R r = sizeof(R) == 4 ? R(__fdividef(float(g[i] - k.eps), float(g[i] - gs[i])))
                                     : (g[i] - k.eps) / (g[i] - gs[i]);
          alpha = r < alpha ? r : alpha;
        }
      }
      alpha = alpha > R(0) ? alpha : R(0);
#pragma unroll
      for (int i = 0; i < Q2; ++i) gs[i] = g[i] + alpha * (gs[i] - g[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < Q2; ++i) g[i] = gs[i];
  return took;
}

struct Grid2 {
  int nx, ny;
  size_t N;
};

// Rows y handled by this thread: y0, y0 + ystride, ...
template <typename R, int VEL>
__global__ void __launch_bounds__(256)
k_step2(const R* __restrict__ in, R* __restrict__ out, Grid2 G, const R* __restrict__ T3,
        const float* __restrict__ u2, int fallback, unsigned long long* __restrict__ counters, const Consts2<R> k) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int ystride = gridDim.y * blockDim.y;
  unsigned took = 0;
  for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < G.ny; y += ystride) {
    if (x >= G.nx) continue;
    const int n = x + G.nx * y;
    // source of velocity component c is coordinate - c
    const int xs[3] = {x + 1 == G.nx ? 0 : x + 1, x, x == 0 ? G.nx - 1 : x - 1};
    const int ys[3] = {(y + 1 == G.ny ? 0 : y + 1) * G.nx, y * G.nx, (y == 0 ? G.ny - 1 : y - 1) * G.nx};
    R g[Q2];
#pragma unroll
    for (int i = 0; i < Q2; ++i) g[i] = __ldg(in + (size_t)i * G.N + (size_t)(xs[cx2(i) + 1] + ys[cy2(i) + 1]));
    R txx = k.txx, txy = k.txy, tyy = k.tyy;
    if (T3 != nullptr) {
      txx = __ldg(T3 + n);
      txy = __ldg(T3 + G.N + n);
      tyy = __ldg(T3 + 2 * G.N + n);
    }
    bool t;
    if constexpr (VEL == 2) {
      const R ux = R(__ldg(u2 + n)), uy = R(__ldg(u2 + G.N + n));
      Consts2<R> kn = k;
      if (ux == R(0) && uy == R(0)) {
        node_tables2(kn, R(0), R(0));
        t = collide2<R, 0>(g, txx, txy, tyy, kn, fallback != 0);
      } else {
        node_tables2(kn, ux, uy);
        t = collide2<R, 1>(g, txx, txy, tyy, kn, fallback != 0);
      }
    } else {
      t = collide2<R, VEL>(g, txx, txy, tyy, k, fallback != 0);
    }
    took += t ? 1u : 0u;
#pragma unroll
    for (int i = 0; i < Q2; ++i) out[(size_t)i * G.N + n] = g[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) took += __shfl_xor_sync(0xffffffffu, took, o);
  if (took != 0u && (threadIdx.x & 31) == 0) atomicAdd(counters, (unsigned long long)took);
}

// Equilibrium of the node's velocity (uniform tables in k, or per node from u2).
template <typename R>
__device__ __forceinline__ R eq_weight(const Consts2<R>& k, const float* u2, size_t N, size_t n, int i) {
  if (u2 == nullptr) return k.E[i];
  const R ux = R(u2[n]), uy = R(u2[N + n]);
  const R cu = R(cx2(i)) * ux + R(cy2(i)) * uy;
  return R(w2(i)) * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * (ux * ux + uy * uy));
}

// Node index of (x + dx, y + dy) with periodic wrap (|dx|, |dy| <= 1).
__device__ __forceinline__ size_t shifted(const Grid2& G, int x, int y, int dx, int dy) {
  x += dx;
  y += dy;
  x = x < 0 ? x + G.nx : (x >= G.nx ? x - G.nx : x);
  y = y < 0 ? y + G.ny : (y >= G.ny ? y - G.ny : y);
  return (size_t)x + (size_t)G.nx * y;
}

// The buffers hold post-collision populations A (the step pulls g_i(x) = A_i(x - c_i)), so a
// pre-collision state g is stored as A_i(y) = g_i(y + c_i).  from_phi: g_i = phi E_i(u), else
// the caller's populations [9][N] (In = float or double).
template <typename R, typename In>
__global__ void k_write2(R* __restrict__ pops, const In* __restrict__ in, Grid2 G, int from_phi,
                         const float* __restrict__ u2, const Consts2<R> k) {
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < G.N; n += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % G.nx), y = (int)(n / G.nx);
#pragma unroll
    for (int i = 0; i < Q2; ++i) {
      const size_t d = shifted(G, x, y, cx2(i), cy2(i));
      pops[(size_t)i * G.N + n] = from_phi ? R(in[d]) * eq_weight(k, u2, G.N, d, i) : R(in[(size_t)i * G.N + d]);
    }
  }
}

// Pre-collision state: what 0: populations g_i(x) = A_i(x - c_i) [9][N]; 1: phi [N]
template <typename R, typename Out>
__global__ void k_read2(const R* __restrict__ pops, Out* __restrict__ out, Grid2 G, int what) {
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < G.N; n += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % G.nx), y = (int)(n / G.nx);
    R s = R(0);
#pragma unroll
    for (int i = 0; i < Q2; ++i) {
      const R v = pops[(size_t)i * G.N + shifted(G, x, y, -cx2(i), -cy2(i))];
      if (what == 0) out[(size_t)i * G.N + n] = Out(v);
      s += v;
    }
    if (what != 0) out[n] = Out(s);
  }
}

constexpr int RED_BLOCKS = 1024;

// FP64 partial sums per block: mass, entropy over positive g, min g, non-finite count.
template <typename R>
__global__ void __launch_bounds__(256) k_reduce2(const R* __restrict__ pops, size_t N, double* __restrict__ part) {
  double m = 0.0, h = 0.0, gmin = 1.7976931348623157e308, bad = 0.0;
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int i = 0; i < Q2; ++i) {
      const double v = (double)pops[(size_t)i * N + n];
      if (!isfinite(v)) {
        bad += 1.0;
        continue;
      }
      m += v;
      if (v > 0.0) h += v * log(v / w2(i));
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
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
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

// Fixed-order sum of the partials (deterministic).
__global__ void k_reduce2_final(const double* __restrict__ part, int nblk, double* __restrict__ out4) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0, b = 0, c = 1.7976931348623157e308, d = 0;
  for (int i = 0; i < nblk; ++i) {
    a += part[4 * i];
    b += part[4 * i + 1];
    c = fmin(c, part[4 * i + 2]);
    d += part[4 * i + 3];
  }
  out4[0] = a;
  out4[1] = b;
  out4[2] = c;
  out4[3] = d;
}

// T = 2I - S = 12 D (I + 6 D)^-1 per node from D3 [3][N] (FP32); counts non-SPD nodes.
template <typename R>
__global__ void k_tensor2(const float* __restrict__ D3, R* __restrict__ T3, size_t N,
                          unsigned long long* __restrict__ bad) {
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    const double a = D3[n], b = D3[N + n], c = D3[2 * N + n];
    if (!(isfinite(a) && isfinite(b) && isfinite(c) && a > 0.0 && a * c - b * b > 0.0)) {
      atomicAdd(bad, 1ull);
      T3[n] = T3[N + n] = T3[2 * N + n] = R(0);
      continue;
    }
    const double m00 = 1.0 + 6.0 * a, m01 = 6.0 * b, m11 = 1.0 + 6.0 * c;
    const double id = 1.0 / (m00 * m11 - m01 * m01);
    const double i00 = m11 * id, i01 = -m01 * id, i11 = m00 * id;
    T3[n] = R(12.0 * (a * i00 + b * i01));
    T3[N + n] = R(12.0 * (a * i01 + b * i11));
    T3[2 * N + n] = R(12.0 * (b * i01 + c * i11));
  }
}

__global__ void k_velocity_check2(const float* __restrict__ u2, size_t N, unsigned long long* __restrict__ bad) {
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    const double ux = u2[n], uy = u2[N + n];
    bool ok = isfinite(ux) && isfinite(uy);
    for (int i = 0; i < Q2 && ok; ++i) {
      const double cu = cx2(i) * ux + cy2(i) * uy;
      ok = 1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy) > 0.0;
    }
    if (!ok) atomicAdd(bad, 1ull);
  }
}

int elementwise_blocks(size_t N) {
  return (int)std::min<size_t>((N + 255) / 256, 152 * 16);
}

bool device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool spd3(const double D[3]) {
  return std::isfinite(D[0]) && std::isfinite(D[1]) && std::isfinite(D[2]) && D[0] > 0 && D[0] * D[2] - D[1] * D[1] > 0;
}

void complement3(const double D[3], double T[3]) {
  const double m00 = 1.0 + 6.0 * D[0], m01 = 6.0 * D[1], m11 = 1.0 + 6.0 * D[2];
  const double id = 1.0 / (m00 * m11 - m01 * m01);
  const double i00 = m11 * id, i01 = -m01 * id, i11 = m00 * id;
  T[0] = 12.0 * (D[0] * i00 + D[1] * i01);
  T[1] = 12.0 * (D[0] * i01 + D[1] * i11);
  T[2] = 12.0 * (D[1] * i01 + D[2] * i11);
}

}  // namespace

struct elbm2d_ctx {
  int nx = 0, ny = 0;
  size_t N = 0;
  int prec = 1;
  cudaStream_t stream = nullptr;
  void* pops[2] = {nullptr, nullptr};
  int cur = 0;
  void* T3 = nullptr;          // per-node T field (R), owned
  float* u2 = nullptr;         // per-node velocity [2][N], owned
  bool have_tensor = false, tensor_field = false;
  double D3[3] = {0, 0, 0};
  double u[2] = {0, 0};
  elbm_params params{};
  Consts2<double> kd{};
  Consts2<float> kf{};
  unsigned long long* d_counters = nullptr;   // [0] fallback count, [1] scratch count
  double* d_part = nullptr;
  double* d_out4 = nullptr;
  bool initialized = false;
  std::string err;
};

namespace {

elbm_status fail(elbm2d_ctx* h, elbm_status s, const std::string& m) {
  if (h) h->err = m;
  return s;
}

elbm_status cuda_fail(elbm2d_ctx* h, cudaError_t e, const char* where) {
  return fail(h, e == cudaErrorMemoryAllocation ? ELBM_ERR_OOM : ELBM_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK2(call, where)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

void rebuild(elbm2d_ctx* h) {
  Consts2<double>& k = h->kd;
  const double ux = h->u[0], uy = h->u[1], uu = ux * ux + uy * uy;
  for (int i = 0; i < Q2; ++i) {
    const double P = poly2(i, ux, uy);
    const double cu = cx2(i) * ux + cy2(i) * uy;
    k.E[i] = w2(i) * P;
    k.K3[i] = 3.0 * (1.0 / P - 1.0);
    k.L[i] = std::log(P) - 3.0 * cu + 1.5 * uu;
    k.M[i] = 1.0 / (w2(i) * P);
  }
  k.ux = ux;
  k.uy = uy;
  k.theta2 = h->params.theta * h->params.theta;
  k.eps = h->params.eps;
  double T[3] = {0, 0, 0};
  if (h->have_tensor && !h->tensor_field) complement3(h->D3, T);
  k.txx = T[0];
  k.txy = T[1];
  k.tyy = T[2];
  Consts2<float>& f = h->kf;
  for (int i = 0; i < Q2; ++i) {
    f.E[i] = (float)k.E[i];
    f.K3[i] = (float)k.K3[i];
    f.L[i] = (float)k.L[i];
    f.M[i] = (float)k.M[i];
  }
  f.ux = (float)k.ux;
  f.uy = (float)k.uy;
  f.theta2 = (float)k.theta2;
  f.eps = (float)k.eps;
  f.txx = (float)k.txx;
  f.txy = (float)k.txy;
  f.tyy = (float)k.tyy;
}

size_t esize(int prec) { return prec == 0 ? 8 : 4; }

// caller array -> device (owned temporary if it was host memory)
elbm_status to_dev(elbm2d_ctx* h, const void* p, size_t bytes, const void** dev, void** tmp) {
  *tmp = nullptr;
  if (device_ptr(p)) {
    *dev = p;
    return ELBM_OK;
  }
  CK2(cudaMallocAsync(tmp, bytes, h->stream), "cudaMallocAsync");
  CK2(cudaMemcpyAsync(*tmp, p, bytes, cudaMemcpyHostToDevice, h->stream), "memcpy H2D");
  *dev = *tmp;
  return ELBM_OK;
}

template <typename R>
cudaError_t launch_step2(elbm2d_ctx* h) {
  const Consts2<R>& k = *reinterpret_cast<const Consts2<R>*>(std::is_same<R, double>::value ? (const void*)&h->kd
                                                                                           : (const void*)&h->kf);
  const int vel = h->u2 ? 2 : ((h->u[0] != 0.0 || h->u[1] != 0.0) ? 1 : 0);
  const int bx = h->nx >= 256 ? 256 : ((h->nx + 31) / 32) * 32;
  const dim3 block(bx, 256 / bx);
  const dim3 grid((h->nx + bx - 1) / bx, (unsigned)std::min<long long>((h->ny + block.y - 1) / block.y, 65535));
  Grid2 G{h->nx, h->ny, h->N};
  const R* in = static_cast<const R*>(h->pops[h->cur]);
  R* out = static_cast<R*>(h->pops[1 - h->cur]);
  const R* T3 = h->tensor_field ? static_cast<const R*>(h->T3) : nullptr;
  const int fb = h->params.fallback;
  if (vel == 2) k_step2<R, 2><<<grid, block, 0, h->stream>>>(in, out, G, T3, h->u2, fb, h->d_counters, k);
  else if (vel == 1) k_step2<R, 1><<<grid, block, 0, h->stream>>>(in, out, G, T3, nullptr, fb, h->d_counters, k);
  else k_step2<R, 0><<<grid, block, 0, h->stream>>>(in, out, G, T3, nullptr, fb, h->d_counters, k);
  return cudaGetLastError();
}

elbm_status write_state(elbm2d_ctx* h, const void* in, elbm_dtype dt, int from_phi) {
  if (!h || !in) return fail(h, ELBM_ERR_ARG, "null argument");
  if (dt != ELBM_DTYPE_F64 && dt != ELBM_DTYPE_F32) return fail(h, ELBM_ERR_ARG, "bad dtype");
  const size_t bytes = (from_phi ? 1 : Q2) * h->N * (dt == ELBM_DTYPE_F64 ? 8 : 4);
  const void* dev;
  void* tmp;
  elbm_status s = to_dev(h, in, bytes, &dev, &tmp);
  if (s != ELBM_OK) return s;
  const int nb = elementwise_blocks(h->N);
  const Grid2 G{h->nx, h->ny, h->N};
  void* p = h->pops[h->cur];
  if (h->prec == 0) {
    if (dt == ELBM_DTYPE_F64)
      k_write2<double, double><<<nb, 256, 0, h->stream>>>((double*)p, (const double*)dev, G, from_phi, h->u2, h->kd);
    else
      k_write2<double, float><<<nb, 256, 0, h->stream>>>((double*)p, (const float*)dev, G, from_phi, h->u2, h->kd);
  } else {
    if (dt == ELBM_DTYPE_F64)
      k_write2<float, double><<<nb, 256, 0, h->stream>>>((float*)p, (const double*)dev, G, from_phi, h->u2, h->kf);
    else
      k_write2<float, float><<<nb, 256, 0, h->stream>>>((float*)p, (const float*)dev, G, from_phi, h->u2, h->kf);
  }
  CK2(cudaGetLastError(), "write kernel");
  if (tmp) CK2(cudaFreeAsync(tmp, h->stream), "cudaFreeAsync");
  CK2(cudaMemsetAsync(h->d_counters, 0, sizeof(unsigned long long), h->stream), "memset");
  h->initialized = true;
  return ELBM_OK;
}

elbm_status read_state(elbm2d_ctx* h, void* out, elbm_dtype dt, int what) {
  if (!h || !out) return fail(h, ELBM_ERR_ARG, "null argument");
  if (!h->initialized) return fail(h, ELBM_ERR_STATE, "state not initialised");
  if (dt != ELBM_DTYPE_F64 && dt != ELBM_DTYPE_F32) return fail(h, ELBM_ERR_ARG, "bad dtype");
  const size_t bytes = (what == 0 ? Q2 : 1) * h->N * (dt == ELBM_DTYPE_F64 ? 8 : 4);
  const bool host = !device_ptr(out);
  void* dout = out;
  if (host) CK2(cudaMallocAsync(&dout, bytes, h->stream), "cudaMallocAsync");
  const int nb = elementwise_blocks(h->N);
  const Grid2 G{h->nx, h->ny, h->N};
  const void* p = h->pops[h->cur];
  if (h->prec == 0) {
    if (dt == ELBM_DTYPE_F64) k_read2<double, double><<<nb, 256, 0, h->stream>>>((const double*)p, (double*)dout, G, what);
    else k_read2<double, float><<<nb, 256, 0, h->stream>>>((const double*)p, (float*)dout, G, what);
  } else {
    if (dt == ELBM_DTYPE_F64) k_read2<float, double><<<nb, 256, 0, h->stream>>>((const float*)p, (double*)dout, G, what);
    else k_read2<float, float><<<nb, 256, 0, h->stream>>>((const float*)p, (float*)dout, G, what);
  }
  CK2(cudaGetLastError(), "read kernel");
  if (host) {
    CK2(cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, h->stream), "memcpy D2H");
    CK2(cudaFreeAsync(dout, h->stream), "cudaFreeAsync");
    CK2(cudaStreamSynchronize(h->stream), "sync");
  }
  return ELBM_OK;
}

}  // namespace

extern "C" {

elbm_status elbm2d_check_velocity(const double u[2]) {
  if (!u) return ELBM_ERR_ARG;
  if (!std::isfinite(u[0]) || !std::isfinite(u[1])) return ELBM_ERR_MACH;
  for (int i = 0; i < Q2; ++i)
    if (!(poly2(i, u[0], u[1]) > 0.0)) return ELBM_ERR_MACH;
  return ELBM_OK;
}

elbm_status elbm2d_relaxation_complement(const double D3[3], double T3_out[3]) {
  if (!D3 || !T3_out) return ELBM_ERR_ARG;
  if (!spd3(D3)) return ELBM_ERR_NOT_SPD;
  complement3(D3, T3_out);
  return ELBM_OK;
}

elbm_status elbm2d_create(const int64_t dims[2], elbm_precision prec, void* cuda_stream, elbm2d_handle* out) {
  if (!dims || !out) return ELBM_ERR_ARG;
  *out = nullptr;
  if ((int)prec < 0 || (int)prec > 3) return ELBM_ERR_ARG;
  if (prec != ELBM_F64 && prec != ELBM_F32) return ELBM_ERR_UNSUPPORTED;
  if (dims[0] < 1 || dims[1] < 1 || dims[0] > 2147483647ll || dims[1] > 2147483647ll) return ELBM_ERR_ARG;
  if ((double)dims[0] * (double)dims[1] >= 2147483647.0) return ELBM_ERR_ARG;
  elbm2d_ctx* h = new elbm2d_ctx();
  h->nx = (int)dims[0];
  h->ny = (int)dims[1];
  h->N = (size_t)dims[0] * (size_t)dims[1];
  h->prec = (int)prec;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->params.theta = prec == ELBM_F64 ? 1e-8 : 3e-4;
  h->params.eps = 0.0;
  h->params.fallback = 1;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&h->pops[b], Q2 * h->N * esize(h->prec));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_counters, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_part, RED_BLOCKS * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_out4, 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_counters, 0, 2 * sizeof(unsigned long long), h->stream);
  if (e != cudaSuccess) {
    const elbm_status s = e == cudaErrorMemoryAllocation ? ELBM_ERR_OOM : ELBM_ERR_CUDA;
    elbm2d_destroy(h);
    return s;
  }
  rebuild(h);
  *out = h;
  return ELBM_OK;
}

void elbm2d_destroy(elbm2d_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->pops[0]);
  cudaFree(h->pops[1]);
  cudaFree(h->T3);
  cudaFree(h->u2);
  cudaFree(h->d_counters);
  cudaFree(h->d_part);
  cudaFree(h->d_out4);
  delete h;
}

const char* elbm2d_last_error(elbm2d_handle h) { return h ? h->err.c_str() : "null handle"; }

elbm_status elbm2d_set_params(elbm2d_handle h, const elbm_params* p) {
  if (!h || !p) return fail(h, ELBM_ERR_ARG, "null argument");
  if (!(p->theta >= 0.0) || !std::isfinite(p->eps)) return fail(h, ELBM_ERR_ARG, "theta must be >= 0, eps finite");
  h->params = *p;
  rebuild(h);
  return ELBM_OK;
}

elbm_status elbm2d_set_tensor_uniform(elbm2d_handle h, const double D3[3]) {
  if (!h || !D3) return fail(h, ELBM_ERR_ARG, "null argument");
  if (!spd3(D3)) return fail(h, ELBM_ERR_NOT_SPD, "tensor is not symmetric positive definite");
  std::memcpy(h->D3, D3, sizeof(h->D3));
  h->have_tensor = true;
  h->tensor_field = false;
  rebuild(h);
  return ELBM_OK;
}

elbm_status elbm2d_set_tensor_field(elbm2d_handle h, const float* D3) {
  if (!h || !D3) return fail(h, ELBM_ERR_ARG, "null argument");
  if (!h->T3) CK2(cudaMalloc(&h->T3, 3 * h->N * esize(h->prec)), "cudaMalloc T field");
  const void* dev;
  void* tmp;
  elbm_status s = to_dev(h, D3, 3 * h->N * sizeof(float), &dev, &tmp);
  if (s != ELBM_OK) return s;
  CK2(cudaMemsetAsync(h->d_counters + 1, 0, sizeof(unsigned long long), h->stream), "memset");
  const int nb = elementwise_blocks(h->N);
  if (h->prec == 0) k_tensor2<double><<<nb, 256, 0, h->stream>>>((const float*)dev, (double*)h->T3, h->N, h->d_counters + 1);
  else k_tensor2<float><<<nb, 256, 0, h->stream>>>((const float*)dev, (float*)h->T3, h->N, h->d_counters + 1);
  CK2(cudaGetLastError(), "tensor pre-pass");
  unsigned long long bad = 0;
  CK2(cudaMemcpyAsync(&bad, h->d_counters + 1, sizeof(bad), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  if (tmp) CK2(cudaFreeAsync(tmp, h->stream), "cudaFreeAsync");
  CK2(cudaStreamSynchronize(h->stream), "sync");
  if (bad) {
    h->have_tensor = false;
    h->tensor_field = false;
    return fail(h, ELBM_ERR_NOT_SPD, std::to_string(bad) + " nodes with a non-SPD or non-finite tensor");
  }
  h->have_tensor = true;
  h->tensor_field = true;
  rebuild(h);
  return ELBM_OK;
}

elbm_status elbm2d_set_velocity_uniform(elbm2d_handle h, const double u[2]) {
  if (!h || !u) return fail(h, ELBM_ERR_ARG, "null argument");
  if (elbm2d_check_velocity(u) != ELBM_OK) return fail(h, ELBM_ERR_MACH, "velocity gives a non-positive P_i(u)");
  if (h->initialized) return fail(h, ELBM_ERR_STATE, "velocity must be set before the state is initialised");
  h->u[0] = u[0];
  h->u[1] = u[1];
  if (h->u2) {
    CK2(cudaStreamSynchronize(h->stream), "sync");
    cudaFree(h->u2);
    h->u2 = nullptr;
  }
  rebuild(h);
  return ELBM_OK;
}

elbm_status elbm2d_set_velocity_field(elbm2d_handle h, const float* u2) {
  if (!h || !u2) return fail(h, ELBM_ERR_ARG, "null argument");
  if (h->initialized) return fail(h, ELBM_ERR_STATE, "velocity must be set before the state is initialised");
  if (!h->u2) CK2(cudaMalloc((void**)&h->u2, 2 * h->N * sizeof(float)), "cudaMalloc velocity field");
  CK2(cudaMemcpyAsync(h->u2, u2, 2 * h->N * sizeof(float), cudaMemcpyDefault, h->stream), "memcpy velocity");
  CK2(cudaMemsetAsync(h->d_counters + 1, 0, sizeof(unsigned long long), h->stream), "memset");
  k_velocity_check2<<<elementwise_blocks(h->N), 256, 0, h->stream>>>(h->u2, h->N, h->d_counters + 1);
  CK2(cudaGetLastError(), "velocity check");
  unsigned long long bad = 0;
  CK2(cudaMemcpyAsync(&bad, h->d_counters + 1, sizeof(bad), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  CK2(cudaStreamSynchronize(h->stream), "sync");
  if (bad) {
    cudaFree(h->u2);
    h->u2 = nullptr;
    return fail(h, ELBM_ERR_MACH, std::to_string(bad) + " nodes whose velocity gives a non-positive P_i(u)");
  }
  h->u[0] = h->u[1] = 0.0;
  rebuild(h);
  return ELBM_OK;
}

elbm_status elbm2d_init_equilibrium(elbm2d_handle h, const void* phi0, elbm_dtype dt) {
  return write_state(h, phi0, dt, 1);
}

elbm_status elbm2d_write_populations(elbm2d_handle h, const void* g, elbm_dtype dt) { return write_state(h, g, dt, 0); }

elbm_status elbm2d_read_populations(elbm2d_handle h, void* out, elbm_dtype dt) { return read_state(h, out, dt, 0); }

elbm_status elbm2d_read_moments(elbm2d_handle h, void* phi, elbm_dtype dt) { return read_state(h, phi, dt, 1); }

elbm_status elbm2d_step(elbm2d_handle h, int64_t nsteps) {
  if (!h) return ELBM_ERR_ARG;
  if (nsteps < 0) return fail(h, ELBM_ERR_ARG, "nsteps < 0");
  if (!h->initialized) return fail(h, ELBM_ERR_STATE, "state not initialised");
  if (!h->have_tensor) return fail(h, ELBM_ERR_STATE, "no diffusion tensor set");
  for (int64_t s = 0; s < nsteps; ++s) {
    CK2(h->prec == 0 ? launch_step2<double>(h) : launch_step2<float>(h), "step kernel");
    h->cur = 1 - h->cur;
  }
  return ELBM_OK;
}

elbm_status elbm2d_reduce(elbm2d_handle h, double* mass, double* entropy, double* gmin, int64_t* n_fallback) {
  if (!h) return ELBM_ERR_ARG;
  if (!h->initialized) return fail(h, ELBM_ERR_STATE, "state not initialised");
  const int nb = (int)std::min<size_t>((h->N + 255) / 256, RED_BLOCKS);
  if (h->prec == 0) k_reduce2<double><<<nb, 256, 0, h->stream>>>((const double*)h->pops[h->cur], h->N, h->d_part);
  else k_reduce2<float><<<nb, 256, 0, h->stream>>>((const float*)h->pops[h->cur], h->N, h->d_part);
  CK2(cudaGetLastError(), "reduce");
  k_reduce2_final<<<1, 32, 0, h->stream>>>(h->d_part, nb, h->d_out4);
  CK2(cudaGetLastError(), "reduce final");
  double o[4];
  unsigned long long fb = 0;
  CK2(cudaMemcpyAsync(o, h->d_out4, sizeof(o), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  CK2(cudaMemcpyAsync(&fb, h->d_counters, sizeof(fb), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  CK2(cudaStreamSynchronize(h->stream), "sync");
  if (mass) *mass = o[0];
  if (entropy) *entropy = o[1];
  if (gmin) *gmin = o[2];
  if (n_fallback) *n_fallback = (int64_t)fb;
  if (o[3] > 0) return fail(h, ELBM_ERR_NONFINITE, std::to_string((long long)o[3]) + " non-finite populations");
  return ELBM_OK;
}

elbm_status elbm2d_synchronize(elbm2d_handle h) {
  if (!h) return ELBM_ERR_ARG;
  CK2(cudaStreamSynchronize(h->stream), "sync");
  CK2(cudaGetLastError(), "async error");
  return ELBM_OK;
}

}  // extern "C"
