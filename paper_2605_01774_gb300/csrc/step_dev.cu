// Fused collide-stream kernel for the deviation storages (FP16 / BF16 deviations,
// FP32 arithmetic).  Same step as k_step (collide.cuh), evaluated in phi-relative
// variables so that the collision produces the stored deviation directly:
//
//   ghat_i = g_i / (W_i phi),  e_i = ghat_i - P_i                (incoming deviation)
//   y_i = e_i - 3 c_i.j',  kappa = sum W_i y_i (K3_i c_i.a' + L_i) / sum (W_i/P_i) y_i^2
//   r_i = g*_i / (W_i phi) - P_i = -kappa e_i + 3 c_i.(a' + kappa j')
//
// with j' = j/phi, a' = a/phi (Eq. method-collision; kappa = lambda - 1 of Eq. method-lambda
// without the identically-zero terms).  Positivity (Eq. method-alpha) in the same
// variables: g*_i < eps  <=>  P_i + r_i < eps/(W_i phi); the quotient
// (g_i - eps)/(g_i - g*_i) = (e_i + P_i - eps/(W_i phi)) / (e_i - r_i); the shortened
// increment gives r_i + (1 - alpha)(e_i - r_i).  Nodes with phi <= 1e-30 take the
// absolute-variable path of collide.cuh.
//
// The FP32 scale plane of the 27 source nodes is staged per 32 x 8 block in shared
// memory (3 z-planes of 34 x 10, periodic wrap resolved at load); the 16-bit deviations
// are read from global memory (each is used once).
#include "internal.h"
#include "pull.cuh"

namespace elbm {

namespace {

constexpr int BX = 32, BY = 8;
constexpr int TX = BX + 2, TY = BY + 2;

// Relative-variable tables: P_i, W_i K3_i, W_i L_i, W_i / P_i (uniform velocity).
struct RelConsts {
  float P[Q];
  float K3W[Q];
  float LW[Q];
  float WP[Q];
};

#ifndef ELBM_DEV_MINB
#define ELBM_DEV_MINB 3
#endif

template <typename Elem, int VEL>
__global__ void __launch_bounds__(256, ELBM_DEV_MINB)
k_step_dev(const Elem* __restrict__ qin, const float* __restrict__ sin, Elem* __restrict__ qout,
           float* __restrict__ sout, Grid G, const float* __restrict__ T6, const float* __restrict__ src, int fallback,
           unsigned long long* __restrict__ counters, const PopConsts<float> k, const RelConsts rc) {
  __shared__ float tile[3][TY][TX];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z = blockIdx.z;
  const int nx = G.nx, ny = G.ny, nz = G.nz, nxy = nx * ny;
  const int N = (int)G.N;
  // stage the scale plane of z-1, z, z+1 for x0-1 .. x0+BX, y0-1 .. y0+BY
  for (int t = ty * BX + tx; t < 3 * TY * TX; t += BX * BY) {
    const int pz = t / (TY * TX), r = t - pz * TY * TX, py = r / TX, px = r - py * TX;
    int gx = x0 - 1 + px, gy = y0 - 1 + py, gz = z - 1 + pz;
    gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
    gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
    gz = gz < 0 ? gz + nz : (gz >= nz ? gz - nz : gz);
    tile[pz][py][px] = (gx < nx && gy < ny) ? __ldg(sin + gx + nx * gy + nxy * gz) : 0.f;
  }
  __syncthreads();
  const int x = x0 + tx, y = y0 + ty;
  bool took = false;
  if (x < nx && y < ny) {
    const int n = x + nx * y + nxy * z;
    const int xs[3] = {x + 1 == nx ? 0 : x + 1, x, x == 0 ? nx - 1 : x - 1};
    const int ys[3] = {(y + 1 == ny ? 0 : y + 1) * nx, y * nx, (y == 0 ? ny - 1 : y - 1) * nx};
    const int zs[3] = {(z + 1 == nz ? 0 : z + 1) * nxy, z * nxy, (z == 0 ? nz - 1 : z - 1) * nxy};
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
      const float s = tile[1 - cz][ty + 1 - cy][tx + 1 - cx];
      const Elem v = __ldg(qin + (i * N + xs[cx + 1] + ys[cy + 1] + zs[cz + 1]));
      g[i] = s * fmaf(float(w_of(i)), Codec<Elem>::to_f(v), k.E[i]);
    }
    if (G.dirichlet && (x == 0 || x == nx - 1)) {
      const float s0 = tile[1][ty + 1][tx + 1];
      if (x == 0) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
          if (cx_of(i) == 1) {
            const int o = opp_of(i);
            const float a = s0 * fmaf(float(w_of(o)), Codec<Elem>::to_f(qin[o * N + n]), k.E[o]);
            g[i] = float(2.0 * w_of(i)) * k.phi_lo - a;
          }
      }
      if (x == nx - 1) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
          if (cx_of(i) == -1) {
            const int o = opp_of(i);
            const float a = s0 * fmaf(float(w_of(o)), Codec<Elem>::to_f(qin[o * N + n]), k.E[o]);
            g[i] = float(2.0 * w_of(i)) * k.phi_hi - a;
          }
      }
    }
    if (src != nullptr) {
      const float r = __ldg(src + n);
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] += r * k.E[i];
    }
    const Sym6<float> T = load_T<float>(T6, G.N, n, k.T);
    float phi, mx, my, mz;
    moments(g, phi, mx, my, mz);
    if (!(phi > 1e-30f)) {
      // absolute-variable path for (nearly) empty nodes
      float ph;
      took = collide_node<float, VEL>(g, T, k, fallback != 0, ph);
      Storage<Elem>::store(qout, sout, N, n, g, k.E, ph);
    } else {
      float jx = mx, jy = my, jz = mz;
      if (VEL == 1) {
        jx = mx - phi * k.ux;
        jy = my - phi * k.uy;
        jz = mz - phi * k.uz;
      }
      float tx_, ty_, tz_;
      sym_mul(T, jx, jy, jz, tx_, ty_, tz_);
      const float inv = 1.0f / phi;
      const float ax = (tx_ - jx) * inv, ay = (ty_ - jy) * inv, az = (tz_ - jz) * inv;   // a'
      const float iw[4] = {inv * float(1.0 / w_of(13)), inv * float(1.0 / w_of(12)), inv * float(1.0 / w_of(9)),
                           inv * float(1.0 / w_of(0))};
      float e[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) e[i] = fmaf(g[i], iw[nnz_of(i)], -rc.P[i]);
      float kappa = 0.f;
      if (VEL == 1) {
        const Dots<float> cj(jx * inv, jy * inv, jz * inv);
        const Dots<float> ca(ax, ay, az);
        float num = 0.f, den = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const float yv = fmaf(-3.0f, cj.d[i], e[i]);
          num = fmaf(yv, fmaf(rc.K3W[i], ca.d[i], rc.LW[i]), num);
          den = fmaf(yv, yv * rc.WP[i], den);
        }
        if (den > k.theta2) kappa = num / den;
      }
      const Dots<float> cb(3.0f * (ax + kappa * jx * inv), 3.0f * (ay + kappa * jy * inv),
                           3.0f * (az + kappa * jz * inv));
      float r[Q];
      bool viol = false;
      const float eh = k.eps;  // eps / (W_i phi) = eps * iw[m]
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        r[i] = fmaf(-kappa, e[i], cb.d[i]);
        viol = viol || (rc.P[i] + r[i] < eh * iw[nnz_of(i)]);
      }
      if (fallback && viol) {
        took = true;
        float alpha = 1.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const float epsh = eh * iw[nnz_of(i)];
          if (rc.P[i] + r[i] < epsh && e[i] > r[i]) {
            const float q = __fdividef(e[i] + rc.P[i] - epsh, e[i] - r[i]);
            alpha = q < alpha ? q : alpha;
          }
        }
        alpha = alpha > 0.f ? alpha : 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) r[i] = fmaf(1.f - alpha, e[i] - r[i], r[i]);
      }
      // encode: q_i = round(r_i); phi_s = phi / (1 + sum W_i q_i) keeps the node mass exactly phi
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const Elem q = Codec<Elem>::from_f(r[i]);
        s = fmaf(float(w_of(i)), Codec<Elem>::to_f(q), s);
        qout[i * N + n] = q;
      }
      sout[n] = phi / (1.0f + s);
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, took);
  if (m != 0u && ((ty * BX + tx) & 31) == 0) atomicAdd(counters, (unsigned long long)__popc(m));
}

template <typename Elem, int VEL>
cudaError_t launch_dev_t(const StepLaunch& L, cudaStream_t s) {
  Grid G{L.nx, L.ny, L.nz, L.N, L.dirichlet};
  RelConsts rc;
  const PopConsts<float>& k = *L.kf;
  const PopConsts<double>& kd = *L.kd;
  for (int i = 0; i < Q; ++i) {
    const double P = kd.E[i] / w_of(i);
    rc.P[i] = (float)P;
    rc.K3W[i] = (float)(w_of(i) * kd.K3[i]);
    rc.LW[i] = (float)(w_of(i) * kd.L[i]);
    rc.WP[i] = (float)(w_of(i) / P);
  }
  dim3 b(BX, BY, 1), g((L.nx + BX - 1) / BX, (L.ny + BY - 1) / BY, L.nz);
  k_step_dev<Elem, VEL><<<g, b, 0, s>>>(static_cast<const Elem*>(L.pin), L.sin, static_cast<Elem*>(L.pout), L.sout, G,
                                        static_cast<const float*>(L.T6), L.src, L.fallback, L.counters, k, rc);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_dev(const StepLaunch& L, cudaStream_t s) {
  const bool v = L.vel != 0;
  if (L.prec == 2) return v ? launch_dev_t<__half, 1>(L, s) : launch_dev_t<__half, 0>(L, s);
  if (L.prec == 3) return v ? launch_dev_t<__nv_bfloat16, 1>(L, s) : launch_dev_t<__nv_bfloat16, 0>(L, s);
  return cudaErrorInvalidValue;
}

}  // namespace elbm
