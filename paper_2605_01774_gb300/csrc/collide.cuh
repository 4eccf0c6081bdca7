// Per-node collision of the anisotropic ADE entropic LBM (Sections 2.2-2.6),
// evaluated in registers on 27 pre-collision populations.
//
// With phi = sum g, j = sum c g - phi u, a = (I - S) j = T j - j (T = 2I - S),
// g_eq_i = phi E_i (E_i = W_i P_i(u)), ds_i = 3 W_i c_i.j, dh_i = g_i - g_eq_i - ds_i,
// the collision of Eq. (method-collision) with amplitude lambda = 1 + kappa is
//     g*_i = g_eq_i + 3 W_i c_i.a - kappa dh_i
//          = (1 + kappa) phi E_i - kappa g_i + 3 W_i c_i.(a + kappa j).
// kappa = lambda - 1 from Eqs. (method-lambda, method-correction) with the terms
// that vanish identically (sum dh = 0, sum c dh = 0) removed:
//     kappa = [sum dh_i K3_i c_i.a + phi sum dh_i L_i] / [sum dh_i^2 M_i],
//     K3_i = 3 (1/P_i - 1), L_i = ln P_i - 3 c_i.u + 1.5 u.u, M_i = 1/(W_i P_i),
// and kappa = 0 where u = 0 (both numerator terms vanish identically), where
// sum dh_i^2 M_i <= theta^2 phi^2 (i.e. <dh|dh>_H <= theta^2 phi), or where phi is not
// above 1e-30 (FP32) / 1e-300 (FP64), below which the H-products are not resolvable.
// The positivity fallback (Eq. method-alpha) shortens g* - g when some g*_i < eps.
#pragma once
#include <type_traits>

#include "eqlog.cuh"
#include "lattice.cuh"

namespace elbm {

// Per-population constants that depend on the uniform velocity (host-computed in FP64).
template <typename R>
struct PopConsts {
  R E[Q];    // W_i P_i(u)
  R Ek[Q];   // E_i 2^e_i (e_i = qexp_of(i)): the equilibrium shape in stored-deviation units
  R K3[Q];   // 3 (1/P_i(u) - 1)
  R L[Q];    // ln P_i(u) - 3 c_i.u + 1.5 u.u
  R M[Q];    // 1 / (W_i P_i(u))
  R ux, uy, uz;
  R theta2;  // theta^2
  R eps;
  R phi_lo, phi_hi;  // Dirichlet wall values
  Sym6<R> T;         // uniform T = 2I - S
  R src_step;        // source multiplier of this step: (a_{n-1} + a_n)/2 (merged Strang halves)
  R src_half;        // half-step multiplier of the stored state: a_{n-1}/2
  int exact_mass;    // FP32 storage: put each node's update rounding back on its rest population
  int root;          // 1: lambda from the exact entropy-stationarity root (FP64 Newton); selects
                     // the ROOT instantiation of the step kernels
};

// Exact root of Eq. (method-entropy-root):
//   f(lam) = sum_i dh_i ln((g_eq_i + ds_post_i + (1 - lam) dh_i) / W_i) = 0.
// With ln(A_i/W_i) = ln phi + ln P_i + log1p(delta_i / g_eq_i), delta_i = ds_post_i + (1 - lam) dh_i,
// and sum dh_i = 0, sum c_i dh_i = 0, the same f is evaluated as
//   f(lam) = sum_i dh_i (L_i + log1p(delta_i / g_eq_i)),  L_i = ln P_i - 3 c_i.u + 1.5 u.u,
// which does not amplify the rounding of sum dh_i by ln phi.  f decreases (f' = -sum dh_i^2/A_i)
// on the open bracket where every A_i > 0.  Safeguarded Newton in FP64 from the closed-form
// lam0; returns lam0 if the bracket is empty.
__device__ __forceinline__ double entropy_root(const double (&geq)[Q], const double (&dsp)[Q], const double (&dh)[Q],
                                               const double (&L)[Q], double lam0) {
  double lo = -1e300, hi = 1e300;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double b = geq[i] + dsp[i];
    if (dh[i] > 0.0) hi = fmin(hi, 1.0 + b / dh[i]);
    else if (dh[i] < 0.0) lo = fmax(lo, 1.0 + b / dh[i]);
    else if (!(b > 0.0)) return lam0;
  }
  if (!(lo < hi)) return lam0;
  double lam = (lam0 > lo && lam0 < hi) ? lam0 : (lo > -1e299 && hi < 1e299 ? 0.5 * (lo + hi) : lam0);
  if (!(lam > lo && lam < hi)) return lam0;
  for (int it = 0; it < 60; ++it) {
    double f = 0.0, fp = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double dl = dsp[i] + (1.0 - lam) * dh[i];
      f += dh[i] * (L[i] + log1p(dl / geq[i]));
      fp -= dh[i] * dh[i] / (geq[i] + dl);
    }
    if (f > 0.0) lo = lam; else hi = lam;
    double nl = lam - f / fp;
    if (!(nl > lo && nl < hi)) nl = (lo > -1e299 && hi < 1e299) ? 0.5 * (lo + hi) : lam0;
    if (fabs(nl - lam) <= 1e-14 * fmax(1.0, fabs(lam))) return nl;
    lam = nl;
  }
  return lam;
}

// c_i . v for all 27 velocities from 9 (cy, cz) partial sums.
template <typename R>
struct Dots {
  R d[Q];
  __device__ __forceinline__ Dots(R vx, R vy, R vz) {
    R yz[9];
#pragma unroll
    for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
      for (int cz = -1; cz <= 1; ++cz) {
        R t = cy == 0 ? R(0) : (cy > 0 ? vy : -vy);
        yz[3 * (cy + 1) + (cz + 1)] = cz == 0 ? t : (cz > 0 ? t + vz : t - vz);
      }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R t = yz[i % 9];
      d[i] = cx_of(i) == 0 ? t : (cx_of(i) > 0 ? t + vx : t - vx);
    }
  }
};

// phi and the first moment sum_i c_i g_i, by partial sums over cz, then cy.
template <typename R>
__device__ __forceinline__ void moments(const R (&g)[Q], R& phi, R& mx, R& my, R& mz) {
  R s[9], dz[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    s[p] = g[3 * p] + g[3 * p + 1] + g[3 * p + 2];
    dz[p] = g[3 * p + 2] - g[3 * p];
  }
  R t[3], e[3];
#pragma unroll
  for (int cx = 0; cx < 3; ++cx) {
    t[cx] = s[3 * cx] + s[3 * cx + 1] + s[3 * cx + 2];
    e[cx] = s[3 * cx + 2] - s[3 * cx];
  }
  phi = t[0] + t[1] + t[2];
  mx = t[2] - t[0];
  my = e[0] + e[1] + e[2];
  mz = (dz[0] + dz[1] + dz[2]) + (dz[3] + dz[4] + dz[5]) + (dz[6] + dz[7] + dz[8]);
}

// P_i(u) tables of one node (per-node velocity fields).
template <typename R>
__device__ __forceinline__ void node_tables(PopConsts<R>& kn, R ux, R uy, R uz) {
  const R uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R cu = R(cx_of(i)) * ux + R(cy_of(i)) * uy + R(cz_of(i)) * uz;
    if constexpr (sizeof(R) == 4) {
      eq_tables_f32(fmaf(3.0f, cu, __fmul_rn(-1.5f, uu)), __fmul_rn(__fmul_rn(4.5f, cu), cu), float(w_of(i)), kn.E[i],
                    kn.K3[i], kn.L[i], kn.M[i]);
    } else {
      const R P = R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu;
      const R rP = R(1) / P;   // one quotient serves K3 and M
      kn.E[i] = R(w_of(i)) * P;
      kn.K3[i] = R(3) * (rP - R(1));
      kn.L[i] = log(P) - R(3) * cu + R(1.5) * uu;
      kn.M[i] = rP * R(1.0 / w_of(i));
    }
  }
  kn.ux = ux;
  kn.uy = uy;
  kn.uz = uz;
}

// VEL = 0: u = 0 exactly (kappa = 0); VEL = 1: uniform u from PopConsts; VEL = 2: the
// node's own velocity un[3] (tables rebuilt per node; lambda = 1 where that u is exactly 0).
// ROOT: lambda from the exact entropy root (k.root); a separate instantiation, so the FP64
// Newton arrays cost the closed-form kernels no registers.
// Returns true if the positivity fallback was taken; phi_out receives the node's phi,
// which the collision conserves exactly.
template <typename R, int VEL, bool ROOT = false>
__device__ __forceinline__ bool collide_node(R (&g)[Q], const Sym6<R>& T, const PopConsts<R>& k,
                                             bool fallback, R& phi_out, const R* un = nullptr) {
  if constexpr (VEL == 2) {
    PopConsts<R> kn = k;
    if (un[0] == R(0) && un[1] == R(0) && un[2] == R(0)) {
      node_tables(kn, R(0), R(0), R(0));
      return collide_node<R, 0>(g, T, kn, fallback, phi_out);
    }
    node_tables(kn, un[0], un[1], un[2]);
    return collide_node<R, 1, ROOT>(g, T, kn, fallback, phi_out);
  }
  R phi, mx, my, mz;
  moments(g, phi, mx, my, mz);
  phi_out = phi;
  R jx = mx, jy = my, jz = mz;
  if (VEL == 1) {
    jx = mx - phi * k.ux;
    jy = my - phi * k.uy;
    jz = mz - phi * k.uz;
  }
  R tx, ty, tz;
  sym_mul(T, jx, jy, jz, tx, ty, tz);
  const R ax = tx - jx, ay = ty - jy, az = tz - jz;  // (I - S) j
  R gs[Q];
  if (VEL == 0) {
    const Dots<R> ca(ax, ay, az);
#pragma unroll
    for (int i = 0; i < Q; ++i) gs[i] = phi * R(w_of(i)) + R(3.0 * w_of(i)) * ca.d[i];
  } else {
    // kappa is a ratio of two sums that are homogeneous of degree 2 in (g, phi, j, a); it is
    // evaluated on the phi-relative quantities dh/phi, j/phi, a/phi, where neither sum can
    // underflow in FP32 and the guard reads sum (dh/phi)^2 M > theta^2.
    R kappa = R(0);
    const R tiny = sizeof(R) == 4 ? R(1e-30) : R(1e-300);
    if (phi > tiny) {
      // FP32: reciprocal-based quotients (2 ulp); inv only normalises the H-products
      const R inv = sizeof(R) == 4 ? R(__fdividef(1.0f, float(phi))) : R(1) / phi;
      const Dots<R> cj(jx * inv, jy * inv, jz * inv);
      const Dots<R> ca(ax * inv, ay * inv, az * inv);
      R num = R(0), den = R(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        R dh = g[i] * inv - k.E[i];
        dh = dh - R(3.0 * w_of(i)) * cj.d[i];
        num += dh * (k.K3[i] * ca.d[i] + k.L[i]);
        den += dh * (dh * k.M[i]);
      }
      if (den > k.theta2) {
        kappa = sizeof(R) == 4 ? R(__fdividef(float(num), float(den))) : num / den;
        if constexpr (ROOT) {
          double geq[Q], dsp[Q], dhd[Q], L[Q];
          const Dots<R> cjd(jx, jy, jz), cad(ax, ay, az);
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            geq[i] = (double)phi * (double)k.E[i];
            dsp[i] = 3.0 * w_of(i) * (double)cad.d[i];
            dhd[i] = (double)g[i] - geq[i] - 3.0 * w_of(i) * (double)cjd.d[i];
            L[i] = (double)k.L[i];
          }
          kappa = R(entropy_root(geq, dsp, dhd, L, 1.0 + (double)kappa) - 1.0);
        }
      }
    }
    const R psi = (R(1) + kappa) * phi;
    const Dots<R> cb(ax + kappa * jx, ay + kappa * jy, az + kappa * jz);
#pragma unroll
    for (int i = 0; i < Q; ++i) gs[i] = psi * k.E[i] - kappa * g[i] + R(3.0 * w_of(i)) * cb.d[i];
  }
  bool took = false;
  if (fallback) {
    bool any = false;
    bool scanned = false;
    if constexpr (sizeof(R) == 8) {
      if (k.eps == R(0)) {
        // FP64 with eps = 0: some g*_i < 0, read from the bit patterns (sign bit set and not
        // -0), so that the test takes integer instructions instead of FP64-pipe compares
        unsigned neg = 0u;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const int hi = __double2hiint(gs[i]);
          const unsigned mag = (unsigned)(hi << 1) | (unsigned)__double2loint(gs[i]);
          neg |= (unsigned)(hi < 0) & (unsigned)(mag != 0u);
        }
        any = neg != 0u;
        scanned = true;
      }
    }
    if (!scanned) {
      // min by fmin (one min instruction per population; a NaN population is skipped, and a
      // NaN node stays NaN whichever way the test goes)
      R mn = gs[0];
#pragma unroll
      for (int i = 1; i < Q; ++i) mn = fmin(mn, gs[i]);
      any = mn < k.eps;
    }
    if (any) {
      took = true;
      // alpha = min over Omega_i < 0 of (g_i - eps) / (-Omega_i), capped at 1.  A ratio is
      // below 1 exactly when g_i + Omega_i < eps, so only the violating populations need a
      // quotient.  gs_i is replaced by d_i = -Omega_i = g_i - g*_i on the way, which the blend
      // g_i + alpha (g*_i - g_i) = g_i - alpha d_i reuses; eps = 0 (the default) is its own
      // loop, without the numerator's subtraction.
      R alpha = R(1);
      auto scan = [&](auto eps0) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const bool viol = gs[i] < k.eps && g[i] > gs[i];
          const R d = g[i] - gs[i];
          if (viol) {
            const R n = decltype(eps0)::value ? g[i] : g[i] - k.eps;
            // FP32: fast reciprocal-based quotient (2 ulp); the rounding of alpha moves the
            // shortened populations by the same order as the FP32 update itself.
            const R r = sizeof(R) == 4 ? R(__fdividef(float(n), float(d))) : n / d;
            alpha = fmin(r, alpha);
          }
          gs[i] = d;
        }
      };
      if (k.eps == R(0)) scan(std::true_type{});
      else scan(std::false_type{});
      alpha = fmax(alpha, R(0));
#pragma unroll
      for (int i = 0; i < Q; ++i) gs[i] = fma(-alpha, gs[i], g[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) g[i] = gs[i];
  return took;
}

}  // namespace elbm
