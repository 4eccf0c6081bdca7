// Hand-written adjoint of the collide-stream step for gradients of a
// concentration misfit with respect to per-node tensor parameters
// theta = (ln d1, ln d2, ln d3, a, b, c):  D = R diag(d) R^T, R = Rz(a) Ry(b) Rz(c),
// T = 2I - S = R diag(t) R^T with t_k = 12 d_k / (1 + 6 d_k)  (Eq. method-s-eigen).
//
// State variable: pre-collision populations G^n [27][N] (periodic lattice, uniform u).
// Forward step (push form of Eq. method-lbe): node y collides G^n(y) and writes
// G^{n+1}_i(y + c_i).  One step's vector-Jacobian product is then a gather:
//   Gbar^n(y) = J_C(G^n(y), T(y))^T [Gbar^{n+1}_i(y + c_i)]_i ,
//   Tbar(y)  += d/dT of the same,
// so every adjoint node update reads its 27 neighbours and writes only its own node: no
// atomics.  (With a pull forward step the transpose would scatter into 27 neighbours.)  The
// push stores are not scattered: for one population a warp writes 32 consecutive nodes shifted
// by c_x, i.e. two 128-byte segments, the same access shape as the pull kernel's loads.
// with the collision of collide.cuh (VEL = 1) differentiated by hand below.
// Misfit J = 1/2 sum_{t in obs} sum_x (phi_t(x) - phi*_t(x))^2, phi_t = sum_i G^t_i,
// enters the reverse sweep as Gbar^t_i(x) += phi_t(x) - phi*_t(x).
// The positivity fallback must stay inactive on gradient runs (its count is returned).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/elbm.h"
#include "../../include/elbm_adjoint.h"
#include "internal.h"

using namespace elbm;

namespace {

struct AGrid {
  int nx, ny, nz;
  int N;
};

__device__ __forceinline__ void coords(const AGrid& G, int n, int& x, int& y, int& z) {
  x = n % G.nx;
  const int r = n / G.nx;
  y = r % G.ny;
  z = r / G.ny;
}

__device__ __forceinline__ int nb(const AGrid& G, int x, int y, int z, int dx, int dy, int dz) {
  x += dx;
  y += dy;
  z += dz;
  x = x < 0 ? x + G.nx : (x >= G.nx ? x - G.nx : x);
  y = y < 0 ? y + G.ny : (y >= G.ny ? y - G.ny : y);
  z = z < 0 ? z + G.nz : (z >= G.nz ? z - G.nz : z);
  return x + G.nx * (y + G.ny * z);
}

template <typename R>
__device__ __forceinline__ R cdot(int i, R vx, R vy, R vz) {
  return R(cx_of(i)) * vx + R(cy_of(i)) * vy + R(cz_of(i)) * vz;
}

// ---------------------------------------------------------------- parameters -> T
template <typename R>
__global__ void k_params_to_T(const R* __restrict__ th, R* __restrict__ T6, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double t[3];
  for (int k = 0; k < 3; ++k) {
    const double d = exp((double)th[k * N + n]);
    t[k] = 12.0 * d / (1.0 + 6.0 * d);
  }
  double sa, ca, sb, cb, sc, cc;
  sincos((double)th[3 * N + n], &sa, &ca);
  sincos((double)th[4 * N + n], &sb, &cb);
  sincos((double)th[5 * N + n], &sc, &cc);
  const double Rm[3][3] = {{ca * cb * cc - sa * sc, -ca * cb * sc - sa * cc, ca * sb},
                           {sa * cb * cc + ca * sc, -sa * cb * sc + ca * cc, sa * sb},
                           {-sb * cc, sb * sc, cb}};
  const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int q = 0; q < 6; ++q) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += Rm[ia[q]][k] * t[k] * Rm[ib[q]][k];
    T6[q * N + n] = (R)s;
  }
}

// dL/dtheta from the accumulated dL/dT (6 unique components, off-diagonals counted once).
template <typename R>
__global__ void k_Tbar_to_params(const R* __restrict__ th, const double* __restrict__ Tbar, R* __restrict__ gth,
                                 int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double d[3], t[3], dt[3];
  for (int k = 0; k < 3; ++k) {
    d[k] = exp((double)th[k * N + n]);
    t[k] = 12.0 * d[k] / (1.0 + 6.0 * d[k]);
    dt[k] = 12.0 * d[k] / ((1.0 + 6.0 * d[k]) * (1.0 + 6.0 * d[k]));  // dt_k / d ln d_k
  }
  // symmetric full-matrix gradient: diagonal as is, off-diagonal halves
  const double g6[6] = {Tbar[n], Tbar[N + n], Tbar[2 * N + n], Tbar[3 * N + n], Tbar[4 * N + n], Tbar[5 * N + n]};
  const double Gm[3][3] = {{g6[0], 0.5 * g6[1], 0.5 * g6[2]},
                           {0.5 * g6[1], g6[3], 0.5 * g6[4]},
                           {0.5 * g6[2], 0.5 * g6[4], g6[5]}};
  const double a = th[3 * N + n], b = th[4 * N + n], c = th[5 * N + n];
  const double sa = sin(a), ca = cos(a), sb = sin(b), cb = cos(b), sc = sin(c), cc = cos(c);
  const double Rz_a[3][3] = {{ca, -sa, 0}, {sa, ca, 0}, {0, 0, 1}};
  const double dRz_a[3][3] = {{-sa, -ca, 0}, {ca, -sa, 0}, {0, 0, 0}};
  const double Ry_b[3][3] = {{cb, 0, sb}, {0, 1, 0}, {-sb, 0, cb}};
  const double dRy_b[3][3] = {{-sb, 0, cb}, {0, 0, 0}, {-cb, 0, -sb}};
  const double Rz_c[3][3] = {{cc, -sc, 0}, {sc, cc, 0}, {0, 0, 1}};
  const double dRz_c[3][3] = {{-sc, -cc, 0}, {cc, -sc, 0}, {0, 0, 0}};
  auto mul = [](const double A[3][3], const double B[3][3], double C[3][3]) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
        C[i][j] = s;
      }
  };
  double tmp[3][3], Q[3][3], dQa[3][3], dQb[3][3], dQc[3][3];
  mul(Rz_a, Ry_b, tmp);
  mul(tmp, Rz_c, Q);
  mul(dRz_a, Ry_b, tmp);
  mul(tmp, Rz_c, dQa);
  mul(Rz_a, dRy_b, tmp);
  mul(tmp, Rz_c, dQb);
  mul(Rz_a, Ry_b, tmp);
  mul(tmp, dRz_c, dQc);
  // dL/dt_k = (Q^T G Q)_kk ; dL/dangle = sum_ab [2 G Q Lambda]_ab dQ_ab
  double GQ[3][3];
  mul(Gm, Q, GQ);
  for (int k = 0; k < 3; ++k) {
    double s = 0;
    for (int i = 0; i < 3; ++i) s += Q[i][k] * GQ[i][k];
    gth[k * N + n] = (R)(s * dt[k]);
  }
  const double(*dQ[3])[3] = {dQa, dQb, dQc};
  for (int m = 0; m < 3; ++m) {
    double s = 0;
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) s += 2.0 * GQ[i][k] * t[k] * dQ[m][i][k];
    gth[(3 + m) * N + n] = (R)s;
  }
}

// ---------------------------------------------------------------- forward (push)
template <typename R>
__global__ void __launch_bounds__(256)
k_adj_forward(const R* __restrict__ Gin, R* __restrict__ Gout, const R* __restrict__ T6, AGrid G,
              const PopConsts<R> k, unsigned long long* fb) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  bool took = false;
  if (n < G.N) {
    R g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = Gin[i * G.N + n];
    const Sym6<R> T{T6[n], T6[G.N + n], T6[2 * G.N + n], T6[3 * G.N + n], T6[4 * G.N + n], T6[5 * G.N + n]};
    R phi;
    took = collide_node<R, 1>(g, T, k, true, phi);
    int x, y, z;
    coords(G, n, x, y, z);
#pragma unroll
    for (int i = 0; i < Q; ++i) Gout[i * G.N + nb(G, x, y, z, cx_of(i), cy_of(i), cz_of(i))] = g[i];
  }
  const unsigned m = __ballot_sync(0xffffffffu, took);
  if (m && (threadIdx.x & 31) == 0) atomicAdd(fb, (unsigned long long)__popc(m));
}

// ---------------------------------------------------------------- one-step VJP
// Gbar_out(y) = J^T gathered adjoint; Tbar(y) += dL/dT (FP64 accumulators); if target
// is given (an observation time), Gbar_out(y)_i += phi(y) - target(y).
template <typename R>
__global__ void __launch_bounds__(256)
k_adj_vjp(const R* __restrict__ Gn, const R* __restrict__ Gbar_next, R* __restrict__ Gbar_out,
          const R* __restrict__ T6, double* __restrict__ Tbar, const R* __restrict__ target, AGrid G,
          const PopConsts<R> k) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= G.N) return;
  int x, y, z;
  coords(G, n, x, y, z);
  R g[Q], yb[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    g[i] = Gn[i * G.N + n];
    yb[i] = Gbar_next[i * G.N + nb(G, x, y, z, cx_of(i), cy_of(i), cz_of(i))];
  }
  const Sym6<R> T{T6[n], T6[G.N + n], T6[2 * G.N + n], T6[3 * G.N + n], T6[4 * G.N + n], T6[5 * G.N + n]};
  // ---- forward recomputation (collide.cuh, VEL = 1, fallback inactive)
  R phi, mx, my, mz;
  moments(g, phi, mx, my, mz);
  const R jx = mx - phi * k.ux, jy = my - phi * k.uy, jz = mz - phi * k.uz;
  R tx, ty, tz;
  sym_mul(T, jx, jy, jz, tx, ty, tz);
  const R ax = tx - jx, ay = ty - jy, az = tz - jz;
  R kappa = R(0), num = R(0), den = R(0), inv = R(0);
  const R tiny = sizeof(R) == 4 ? R(1e-30) : R(1e-300);
  const bool kap_on_phi = phi > tiny;
  if (kap_on_phi) {
    inv = R(1) / phi;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R dh = g[i] * inv - k.E[i] - R(3.0 * w_of(i)) * cdot<R>(i, jx * inv, jy * inv, jz * inv);
      num += dh * (k.K3[i] * cdot<R>(i, ax * inv, ay * inv, az * inv) + k.L[i]);
      den += dh * dh * k.M[i];
    }
  }
  const bool kap_on = kap_on_phi && den > k.theta2;
  if (kap_on) kappa = num / den;
  // ---- reverse
  R psib = R(0), kapb = R(0), bbx = R(0), bby = R(0), bbz = R(0);
  R gb[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    psib += yb[i] * k.E[i];
    kapb -= yb[i] * g[i];
    gb[i] = -kappa * yb[i];
    const R w3 = R(3.0 * w_of(i)) * yb[i];
    bbx += R(cx_of(i)) * w3;
    bby += R(cy_of(i)) * w3;
    bbz += R(cz_of(i)) * w3;
  }
  // psi = (1 + kappa) phi ; b = a + kappa j
  kapb += psib * phi;
  R phib = psib * (R(1) + kappa);
  R abx = bbx, aby = bby, abz = bbz;
  kapb += bbx * jx + bby * jy + bbz * jz;
  R jbx = kappa * bbx, jby = kappa * bby, jbz = kappa * bbz;
  if (kap_on) {
    const R numb = kapb / den;
    const R denb = -kapb * kappa / den;
    R apbx = R(0), apby = R(0), apbz = R(0), jpbx = R(0), jpby = R(0), jpbz = R(0), invb = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R cj = cdot<R>(i, jx * inv, jy * inv, jz * inv);
      const R ca = cdot<R>(i, ax * inv, ay * inv, az * inv);
      const R dh = g[i] * inv - k.E[i] - R(3.0 * w_of(i)) * cj;
      const R t = k.K3[i] * ca + k.L[i];
      const R dhb = numb * t + R(2) * denb * dh * k.M[i];
      const R cak = numb * dh * k.K3[i];            // d num / d (c_i . a')
      apbx += R(cx_of(i)) * cak;
      apby += R(cy_of(i)) * cak;
      apbz += R(cz_of(i)) * cak;
      gb[i] += dhb * inv;
      invb += dhb * g[i];
      const R cjb = -dhb * R(3.0 * w_of(i));        // d / d (c_i . j')
      jpbx += R(cx_of(i)) * cjb;
      jpby += R(cy_of(i)) * cjb;
      jpbz += R(cz_of(i)) * cjb;
    }
    // a' = a inv ; j' = j inv ; inv = 1 / phi
    abx += apbx * inv;
    aby += apby * inv;
    abz += apbz * inv;
    invb += apbx * ax + apby * ay + apbz * az;
    jbx += jpbx * inv;
    jby += jpby * inv;
    jbz += jpbz * inv;
    invb += jpbx * jx + jpby * jy + jpbz * jz;
    phib -= invb * inv * inv;
  }
  // a = T j - j
  R Tax, Tay, Taz;
  sym_mul(T, abx, aby, abz, Tax, Tay, Taz);
  jbx += Tax - abx;
  jby += Tay - aby;
  jbz += Taz - abz;
  Tbar[n] += (double)(abx * jx);
  Tbar[G.N + n] += (double)(abx * jy + aby * jx);
  Tbar[2 * G.N + n] += (double)(abx * jz + abz * jx);
  Tbar[3 * G.N + n] += (double)(aby * jy);
  Tbar[4 * G.N + n] += (double)(aby * jz + abz * jy);
  Tbar[5 * G.N + n] += (double)(abz * jz);
  // j = m - phi u ; m = sum c g ; phi = sum g
  phib -= k.ux * jbx + k.uy * jby + k.uz * jbz;
  R inj = R(0);
  if (target != nullptr) inj = phi - target[n];
#pragma unroll
  for (int i = 0; i < Q; ++i)
    Gbar_out[i * G.N + n] = gb[i] + R(cx_of(i)) * jbx + R(cy_of(i)) * jby + R(cz_of(i)) * jbz + phib + inj;
}

// misfit contribution 1/2 sum (phi - target)^2 and phi-adjoint seed at the last step
template <typename R>
__global__ void __launch_bounds__(256)
k_adj_misfit(const R* __restrict__ Gs, const R* __restrict__ target, double* __restrict__ part, R* __restrict__ seed,
             int N) {
  __shared__ double sm[256];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (n < N) {
    R phi = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) phi += Gs[i * N + n];
    const double d = (double)phi - (double)target[n];
    v = 0.5 * d * d;
    if (seed != nullptr) {
#pragma unroll
      for (int i = 0; i < Q; ++i) seed[i * N + n] += (R)d;
    }
  }
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

}  // namespace

struct elbm_adjoint_ctx {
  AGrid G{};
  int prec = 0;
  cudaStream_t stream = nullptr;
  double u[3] = {0, 0, 0};
  double theta = 1e-8;
  int K = 50;
  PopConsts<double> kd{};
  PopConsts<float> kf{};
  void* T6 = nullptr;              // [6][N] R
  double* Tbar = nullptr;          // [6][N]
  void* ck = nullptr;              // checkpoints, allocated per run
  void* seg = nullptr;             // segment states
  void* gbar[2] = {nullptr, nullptr};
  double* part = nullptr;
  unsigned long long* fb = nullptr;
  std::string err;
};

namespace {

elbm_status afail(elbm_adjoint_ctx* h, elbm_status s, const std::string& m) {
  if (h) h->err = m;
  return s;
}
#define ACK(call, where)                                                                           \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return afail(h, e_ == cudaErrorMemoryAllocation ? ELBM_ERR_OOM : ELBM_ERR_CUDA,              \
                   std::string(where) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

void consts_for(elbm_adjoint_ctx* h) {
  const double* u = h->u;
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  PopConsts<double>& k = h->kd;
  for (int i = 0; i < Q; ++i) {
    const double cu = cx_of(i) * u[0] + cy_of(i) * u[1] + cz_of(i) * u[2];
    const double P = 1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu;
    k.E[i] = w_of(i) * P;
    k.K3[i] = 3.0 * (1.0 / P - 1.0);
    k.L[i] = std::log(P) - 3.0 * cu + 1.5 * uu;
    k.M[i] = 1.0 / (w_of(i) * P);
  }
  k.ux = u[0];
  k.uy = u[1];
  k.uz = u[2];
  k.theta2 = h->theta * h->theta;
  k.eps = 0.0;
  PopConsts<float>& f = h->kf;
  for (int i = 0; i < Q; ++i) {
    f.E[i] = (float)k.E[i];
    f.K3[i] = (float)k.K3[i];
    f.L[i] = (float)k.L[i];
    f.M[i] = (float)k.M[i];
  }
  f.ux = (float)u[0];
  f.uy = (float)u[1];
  f.uz = (float)u[2];
  f.theta2 = (float)k.theta2;
  f.eps = 0.f;
}

template <typename R>
const PopConsts<R>& kc(elbm_adjoint_ctx* h);
template <>
const PopConsts<double>& kc<double>(elbm_adjoint_ctx* h) {
  return h->kd;
}
template <>
const PopConsts<float>& kc<float>(elbm_adjoint_ctx* h) {
  return h->kf;
}

int blocks(int N) { return (N + 255) / 256; }

template <typename R>
__global__ void k_adj_init(const R* __restrict__ phi0, R* __restrict__ Gs, int N, const PopConsts<R> k) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const R p = phi0[n];
#pragma unroll
  for (int i = 0; i < Q; ++i) Gs[i * N + n] = p * k.E[i];
}

template <typename R>
elbm_status run_t(elbm_adjoint_ctx* h, const R* theta, const R* phi0, int64_t nsteps, int nobs, const int64_t* obs,
                  const R* targets, double* J, R* grad, int64_t* nfb) {
  const AGrid G = h->G;
  const int N = G.N;
  const size_t sb = 27ull * N * sizeof(R);
  const int K = h->K;
  const int nck = (int)(nsteps / K) + 1;
  cudaStream_t s = h->stream;
  const PopConsts<R>& k = kc<R>(h);
  k_params_to_T<R><<<blocks(N), 256, 0, s>>>(theta, static_cast<R*>(h->T6), N);
  ACK(cudaGetLastError(), "params");
  R* ck = nullptr;
  R* seg = nullptr;
  ACK(cudaMallocAsync((void**)&ck, sb * nck, s), "checkpoint buffer");
  ACK(cudaMallocAsync((void**)&seg, sb * (size_t)(K + 1), s), "segment buffer");
  const R* T6 = static_cast<const R*>(h->T6);
  ACK(cudaMemsetAsync(h->fb, 0, sizeof(unsigned long long), s), "memset");
  ACK(cudaMemsetAsync(h->part, 0, sizeof(double) * blocks(N) * (nobs + 1), s), "memset");
  auto obs_index = [&](int64_t t) {
    for (int o = 0; o < nobs; ++o)
      if (obs[o] == t) return o;
    return -1;
  };
  // forward sweep: checkpoints every K steps, misfit at the observation steps
  k_adj_init<R><<<blocks(N), 256, 0, s>>>(phi0, ck, N, k);
  ACK(cudaGetLastError(), "init");
  R* cur = ck;          // state G^t
  R* nxt = seg;         // scratch for the next state when not a checkpoint
  for (int64_t t = 0; t < nsteps; ++t) {
    R* dst = ((t + 1) % K == 0) ? ck + 27ull * N * ((t + 1) / K) : (cur == seg ? seg + 27ull * N : seg);
    k_adj_forward<R><<<blocks(N), 256, 0, s>>>(cur, dst, T6, G, k, h->fb);
    ACK(cudaGetLastError(), "forward");
    cur = dst;
    const int o = obs_index(t + 1);
    if (o >= 0) {
      k_adj_misfit<R><<<blocks(N), 256, 0, s>>>(cur, targets + (size_t)o * N, h->part + (size_t)o * blocks(N),
                                               nullptr, N);
      ACK(cudaGetLastError(), "misfit");
    }
  }
  (void)nxt;
  std::vector<double> part((size_t)blocks(N) * nobs);
  ACK(cudaMemcpyAsync(part.data(), h->part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "memcpy");
  unsigned long long fb = 0;
  ACK(cudaMemcpyAsync(&fb, h->fb, sizeof(fb), cudaMemcpyDeviceToHost, s), "memcpy");
  ACK(cudaStreamSynchronize(s), "sync");
  double Jv = 0.0;
  for (double v : part) Jv += v;
  if (J) *J = Jv;
  if (nfb) *nfb = (int64_t)fb;
  if (grad != nullptr) {
    // reverse sweep, segment by segment from the end
    R* gb0 = static_cast<R*>(h->gbar[0]);
    R* gb1 = static_cast<R*>(h->gbar[1]);
    ACK(cudaMemsetAsync(gb0, 0, sb, s), "memset");
    ACK(cudaMemsetAsync(h->Tbar, 0, 6ull * N * sizeof(double), s), "memset");
    const int o_last = obs_index(nsteps);
    if (o_last >= 0) {
      // seed: Gbar^T_i = phi_T - target (recompute G^T into seg[0..])
      const int64_t t0 = (nsteps / K) * K;
      R* st = ck + 27ull * N * (t0 / K);
      for (int64_t t = t0; t < nsteps; ++t) {
        R* dst = seg + 27ull * N * ((t - t0) % 2);
        k_adj_forward<R><<<blocks(N), 256, 0, s>>>(st, dst, T6, G, k, h->fb);
        st = dst;
      }
      k_adj_misfit<R><<<blocks(N), 256, 0, s>>>(st, targets + (size_t)o_last * N,
                                               h->part + (size_t)nobs * blocks(N), gb0, N);
      ACK(cudaGetLastError(), "seed");
    }
    R* gin = gb0;   // Gbar^{t+1}
    R* gout = gb1;  // Gbar^t
    for (int64_t sgm = (nsteps - 1) / K; sgm >= 0; --sgm) {
      const int64_t t0 = sgm * K;
      const int64_t t1 = std::min<int64_t>(nsteps, t0 + K);
      // recompute G^{t0 .. t1-1} into seg[0 .. t1-t0-1]
      ACK(cudaMemcpyAsync(seg, ck + 27ull * N * sgm, sb, cudaMemcpyDeviceToDevice, s), "memcpy");
      for (int64_t t = t0; t < t1 - 1; ++t) {
        k_adj_forward<R><<<blocks(N), 256, 0, s>>>(seg + 27ull * N * (t - t0), seg + 27ull * N * (t - t0 + 1), T6,
                                                  G, k, h->fb);
      }
      ACK(cudaGetLastError(), "recompute");
      for (int64_t t = t1 - 1; t >= t0; --t) {
        const int o = obs_index(t);
        const R* tgt = (o >= 0 && t > 0) ? targets + (size_t)o * N : nullptr;
        k_adj_vjp<R><<<blocks(N), 256, 0, s>>>(seg + 27ull * N * (t - t0), gin, gout, T6, h->Tbar, tgt, G, k);
        std::swap(gin, gout);
      }
      ACK(cudaGetLastError(), "vjp");
    }
    k_Tbar_to_params<R><<<blocks(N), 256, 0, s>>>(theta, h->Tbar, grad, N);
    ACK(cudaGetLastError(), "chain rule");
  }
  ACK(cudaFreeAsync(ck, s), "free");
  ACK(cudaFreeAsync(seg, s), "free");
  ACK(cudaStreamSynchronize(s), "sync");
  return ELBM_OK;
}

}  // namespace

extern "C" {

elbm_status elbm_adjoint_create(const int64_t dims[3], elbm_precision prec, void* cuda_stream,
                                elbm_adjoint_handle* out) {
  if (!dims || !out) return ELBM_ERR_ARG;
  *out = nullptr;
  if (prec != ELBM_F64 && prec != ELBM_F32) return ELBM_ERR_UNSUPPORTED;
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 1 || dims[a] > 4096) return ELBM_ERR_ARG;
  const double N = (double)dims[0] * dims[1] * dims[2];
  if (27.0 * N >= 2147483647.0) return ELBM_ERR_ARG;
  elbm_adjoint_ctx* h = new elbm_adjoint_ctx();
  h->G = AGrid{(int)dims[0], (int)dims[1], (int)dims[2], (int)N};
  h->prec = (int)prec;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  const size_t rs = prec == ELBM_F64 ? 8 : 4;
  cudaError_t e = cudaMalloc(&h->T6, 6 * (size_t)N * rs);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->Tbar, 6 * (size_t)N * sizeof(double));
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&h->gbar[b], 27 * (size_t)N * rs);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->fb, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->part, sizeof(double) * blocks((int)N) * 17);
  if (e != cudaSuccess) {
    elbm_adjoint_destroy(h);
    return e == cudaErrorMemoryAllocation ? ELBM_ERR_OOM : ELBM_ERR_CUDA;
  }
  consts_for(h);
  *out = h;
  return ELBM_OK;
}

void elbm_adjoint_destroy(elbm_adjoint_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->T6);
  cudaFree(h->Tbar);
  cudaFree(h->gbar[0]);
  cudaFree(h->gbar[1]);
  cudaFree(h->fb);
  cudaFree(h->part);
  delete h;
}

const char* elbm_adjoint_last_error(elbm_adjoint_handle h) { return h ? h->err.c_str() : "null handle"; }

elbm_status elbm_adjoint_configure(elbm_adjoint_handle h, const double u[3], double theta, int32_t checkpoint_every) {
  if (!h || !u || !(theta >= 0.0) || checkpoint_every < 1) return afail(h, ELBM_ERR_ARG, "bad argument");
  if (elbm_check_velocity(u) != ELBM_OK) return afail(h, ELBM_ERR_MACH, "velocity gives a non-positive P_i(u)");
  std::memcpy(h->u, u, sizeof(h->u));
  h->theta = theta;
  h->K = checkpoint_every;
  consts_for(h);
  return ELBM_OK;
}

elbm_status elbm_adjoint_misfit(elbm_adjoint_handle h, const void* theta6, const void* phi0, int64_t nsteps,
                                int32_t nobs, const int64_t* obs_steps, const void* targets, double* J, void* grad6,
                                int64_t* n_fallback) {
  if (!h || !theta6 || !phi0 || nsteps < 1 || nobs < 1 || nobs > 16 || !obs_steps || !targets)
    return afail(h, ELBM_ERR_ARG, "bad argument");
  for (int o = 0; o < nobs; ++o)
    if (obs_steps[o] < 1 || obs_steps[o] > nsteps) return afail(h, ELBM_ERR_ARG, "observation step out of range");
  if (h->prec == ELBM_F64)
    return run_t<double>(h, (const double*)theta6, (const double*)phi0, nsteps, nobs, obs_steps,
                         (const double*)targets, J, (double*)grad6, n_fallback);
  return run_t<float>(h, (const float*)theta6, (const float*)phi0, nsteps, nobs, obs_steps, (const float*)targets, J,
                      (float*)grad6, n_fallback);
}

}  // extern "C"

template <typename R>
static elbm_status step_t(elbm_adjoint_ctx* h, const R* theta, const R* g, const R* gbar_next, R* g_next, R* gbar,
                          R* grad) {
  const int N = h->G.N;
  cudaStream_t s = h->stream;
  k_params_to_T<R><<<blocks(N), 256, 0, s>>>(theta, static_cast<R*>(h->T6), N);
  ACK(cudaGetLastError(), "params");
  if (g_next) {
    k_adj_forward<R><<<blocks(N), 256, 0, s>>>(g, g_next, static_cast<const R*>(h->T6), h->G, kc<R>(h), h->fb);
    ACK(cudaGetLastError(), "forward");
  }
  if (gbar) {
    ACK(cudaMemsetAsync(h->Tbar, 0, 6ull * N * sizeof(double), s), "memset");
    k_adj_vjp<R><<<blocks(N), 256, 0, s>>>(g, gbar_next, gbar, static_cast<const R*>(h->T6), h->Tbar, nullptr, h->G,
                                          kc<R>(h));
    ACK(cudaGetLastError(), "vjp");
    if (grad) {
      k_Tbar_to_params<R><<<blocks(N), 256, 0, s>>>(theta, h->Tbar, grad, N);
      ACK(cudaGetLastError(), "chain rule");
    }
  }
  ACK(cudaStreamSynchronize(s), "sync");
  return ELBM_OK;
}

extern "C" {

elbm_status elbm_adjoint_step(elbm_adjoint_handle h, const void* theta6, const void* g, const void* gbar_next,
                              void* g_next, void* gbar, void* grad6) {
  if (!h || !theta6 || !g || (gbar && !gbar_next)) return afail(h, ELBM_ERR_ARG, "bad argument");
  if (h->prec == ELBM_F64)
    return step_t<double>(h, (const double*)theta6, (const double*)g, (const double*)gbar_next, (double*)g_next,
                          (double*)gbar, (double*)grad6);
  return step_t<float>(h, (const float*)theta6, (const float*)g, (const float*)gbar_next, (float*)g_next,
                       (float*)gbar, (float*)grad6);
}

}  // extern "C"
