// C ABI (include/elbm.h): handle management, argument checks, host/device
// marshalling and the launch sequence of the single-lattice path.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/elbm.h"
#include "internal.h"

using namespace elbm;

struct elbm_ctx {
  int nx = 0, ny = 0, nz = 0;
  size_t N = 0;
  int prec = 1;
  elbm_bc bc{};
  cudaStream_t stream = nullptr;
  int device = 0;
  void* pops[2] = {nullptr, nullptr};
  float* scale[2] = {nullptr, nullptr};
  int cur = 0;
  void* T6 = nullptr;        // per-node T field (owned; double for FP64, else float)
  float* src = nullptr;      // per-node source (owned)
  float* u3 = nullptr;       // per-node velocity [3][N] (owned), null = uniform u
  bool have_tensor = false;
  bool tensor_field = false;
  double D6[6] = {0, 0, 0, 0, 0, 0};
  double u[3] = {0, 0, 0};
  elbm_params params{};
  PopConsts<double> kd{};
  PopConsts<float> kf{};
  unsigned long long* d_counters = nullptr;
  double* d_scratch = nullptr;
  double* d_out4 = nullptr;
  int64_t step = 0;
  bool initialized = false;
  double src_amp = 1.0;      // source amplitude of the most recent half-step a_{n-1}
  int lambda_mode = 0;       // 0 closed form, 1 exact root
  int step_kernel = 0;       // 0 auto, 1 per-node gathers, 2 staged rows, 3 pipelined staged rows
  long long wait_limit = 0;  // staging-wait limit in clock cycles (0: the default, about one second)
  int wait_withheld = 0;      // test hook: arrivals the staged-row barriers expect and never get
  int exact_mass = 1;        // FP32 storage: exact stored node mass
  std::string err;
};

namespace {

size_t elem_size(int prec) { return prec == 0 ? 8 : prec == 1 ? 4 : 2; }
bool is_dev_format(int prec) { return prec >= 2; }

elbm_status fail(elbm_ctx* h, elbm_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

elbm_status cuda_fail(elbm_ctx* h, cudaError_t e, const char* where) {
  return fail(h, e == cudaErrorMemoryAllocation ? ELBM_ERR_OOM : ELBM_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Symmetric 3x3 helpers on (xx, xy, xz, yy, yz, zz).
double det6(const double m[6]) {
  return m[0] * (m[3] * m[5] - m[4] * m[4]) - m[1] * (m[1] * m[5] - m[4] * m[2]) + m[2] * (m[1] * m[4] - m[3] * m[2]);
}
bool spd6(const double D[6]) {
  for (int q = 0; q < 6; ++q)
    if (!std::isfinite(D[q])) return false;
  return D[0] > 0 && D[0] * D[3] - D[1] * D[1] > 0 && det6(D) > 0;
}
void inv6(const double m[6], double o[6]) {
  const double a = m[0], b = m[1], c = m[2], d = m[3], e = m[4], f = m[5];
  const double A = d * f - e * e, B = c * e - b * f, C = b * e - c * d;
  const double id = 1.0 / (a * A + b * B + c * C);
  o[0] = A * id;
  o[1] = B * id;
  o[2] = C * id;
  o[3] = (a * f - c * c) * id;
  o[4] = (b * c - a * e) * id;
  o[5] = (a * d - b * b) * id;
}
// T = 2I - S = 12 D (I + 6 D)^-1 (Eq. method-s-from-d, cs2 = 1/3, dt = 1)
void complement6(const double D[6], double T[6]) {
  const double M[6] = {1 + 6 * D[0], 6 * D[1], 6 * D[2], 1 + 6 * D[3], 6 * D[4], 1 + 6 * D[5]};
  double Mi[6];
  inv6(M, Mi);
  const double Dm[3][3] = {{D[0], D[1], D[2]}, {D[1], D[3], D[4]}, {D[2], D[4], D[5]}};
  const double Im[3][3] = {{Mi[0], Mi[1], Mi[2]}, {Mi[1], Mi[3], Mi[4]}, {Mi[2], Mi[4], Mi[5]}};
  const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int q = 0; q < 6; ++q) {
    double s = 0;
    for (int k = 0; k < 3; ++k) s += Dm[ia[q]][k] * Im[k][ib[q]];
    T[q] = 12.0 * s;
  }
}

double poly_of(int i, const double u[3]) {
  const double cu = cx_of(i) * u[0] + cy_of(i) * u[1] + cz_of(i) * u[2];
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return 1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu;
}

// Per-population tables of collide.cuh, in FP64 then rounded for the FP32 kernels.
void rebuild_consts(elbm_ctx* h) {
  PopConsts<double>& k = h->kd;
  const double* u = h->u;
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    const double P = poly_of(i, u);
    const double cu = cx_of(i) * u[0] + cy_of(i) * u[1] + cz_of(i) * u[2];
    k.E[i] = w_of(i) * P;
    k.Ek[i] = std::ldexp(k.E[i], qexp_of(i));
    k.K3[i] = 3.0 * (1.0 / P - 1.0);
    k.L[i] = std::log(P) - 3.0 * cu + 1.5 * uu;
    k.M[i] = 1.0 / (w_of(i) * P);
  }
  k.ux = u[0];
  k.uy = u[1];
  k.uz = u[2];
  k.theta2 = h->params.theta * h->params.theta;
  k.eps = h->params.eps;
  k.phi_lo = h->bc.phi_lo;
  k.phi_hi = h->bc.phi_hi;
  k.src_step = h->src_amp;
  k.src_half = 0.5 * h->src_amp;
  k.root = h->lambda_mode;
  k.exact_mass = h->exact_mass;
  double T[6] = {0, 0, 0, 0, 0, 0};
  if (h->have_tensor && !h->tensor_field) complement6(h->D6, T);
  k.T = Sym6<double>{T[0], T[1], T[2], T[3], T[4], T[5]};
  PopConsts<float>& f = h->kf;
  for (int i = 0; i < Q; ++i) {
    f.E[i] = (float)k.E[i];
    f.Ek[i] = (float)k.Ek[i];
    f.K3[i] = (float)k.K3[i];
    f.L[i] = (float)k.L[i];
    f.M[i] = (float)k.M[i];
  }
  f.ux = (float)k.ux;
  f.uy = (float)k.uy;
  f.uz = (float)k.uz;
  f.theta2 = (float)k.theta2;
  f.eps = (float)k.eps;
  f.phi_lo = (float)k.phi_lo;
  f.phi_hi = (float)k.phi_hi;
  f.src_step = (float)k.src_step;
  f.src_half = (float)k.src_half;
  f.root = k.root;
  f.exact_mass = k.exact_mass;
  f.T = Sym6<float>{(float)T[0], (float)T[1], (float)T[2], (float)T[3], (float)T[4], (float)T[5]};
}

StateIO state_io(elbm_ctx* h) {
  StateIO S;
  S.prec = h->prec;
  S.nx = h->nx;
  S.ny = h->ny;
  S.nz = h->nz;
  S.N = h->N;
  S.dirichlet = h->bc.dirichlet_x;
  S.pops = h->pops[h->cur];
  S.scale = h->scale[h->cur];
  S.T6 = h->tensor_field ? h->T6 : nullptr;
  S.u3 = h->u3;
  S.src = h->src;
  S.kd = &h->kd;
  S.kf = &h->kf;
  return S;
}

// Bring a caller array of `bytes` to the device; *tmp receives an owned copy if it was on the host.
elbm_status to_device(elbm_ctx* h, const void* p, size_t bytes, const void** dev, void** tmp) {
  *tmp = nullptr;
  if (is_device_ptr(p)) {
    *dev = p;
    return ELBM_OK;
  }
  CK(cudaMallocAsync(tmp, bytes, h->stream), "cudaMallocAsync");
  CK(cudaMemcpyAsync(*tmp, p, bytes, cudaMemcpyHostToDevice, h->stream), "cudaMemcpyAsync H2D");
  *dev = *tmp;
  return ELBM_OK;
}

}  // namespace

extern "C" {

const char* elbm_status_string(elbm_status s) {
  switch (s) {
    case ELBM_OK: return "ELBM_OK";
    case ELBM_ERR_ARG: return "ELBM_ERR_ARG";
    case ELBM_ERR_NOT_SPD: return "ELBM_ERR_NOT_SPD";
    case ELBM_ERR_MACH: return "ELBM_ERR_MACH";
    case ELBM_ERR_OOM: return "ELBM_ERR_OOM";
    case ELBM_ERR_CUDA: return "ELBM_ERR_CUDA";
    case ELBM_ERR_NONFINITE: return "ELBM_ERR_NONFINITE";
    case ELBM_ERR_TIMEOUT: return "ELBM_ERR_TIMEOUT";
    case ELBM_ERR_STATE: return "ELBM_ERR_STATE";
    case ELBM_ERR_UNSUPPORTED: return "ELBM_ERR_UNSUPPORTED";
  }
  return "unknown";
}

elbm_status elbm_check_tensor(const double D6[6]) {
  if (!D6) return ELBM_ERR_ARG;
  return spd6(D6) ? ELBM_OK : ELBM_ERR_NOT_SPD;
}

elbm_status elbm_check_velocity(const double u[3]) {
  if (!u) return ELBM_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(u[k])) return ELBM_ERR_MACH;
  for (int i = 0; i < Q; ++i)
    if (!(poly_of(i, u) > 0.0)) return ELBM_ERR_MACH;
  return ELBM_OK;
}

elbm_status elbm_relaxation_complement(const double D6[6], double T6_out[6]) {
  if (!D6 || !T6_out) return ELBM_ERR_ARG;
  if (!spd6(D6)) return ELBM_ERR_NOT_SPD;
  complement6(D6, T6_out);
  return ELBM_OK;
}

elbm_status elbm_create(const int64_t dims[3], elbm_precision prec, const elbm_bc* bc, void* cuda_stream,
                        elbm_handle* out) {
  if (!dims || !out) return ELBM_ERR_ARG;
  *out = nullptr;
  if ((int)prec < 0 || (int)prec > 3) return ELBM_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 1 || dims[a] > 65535) return ELBM_ERR_ARG;
  const double N = (double)dims[0] * (double)dims[1] * (double)dims[2];
  if (27.0 * N >= 2147483647.0) return ELBM_ERR_ARG;
  if (bc && bc->dirichlet_x != 0 && bc->dirichlet_x != 1) return ELBM_ERR_ARG;
  elbm_ctx* h = new elbm_ctx();
  h->nx = (int)dims[0];
  h->ny = (int)dims[1];
  h->nz = (int)dims[2];
  h->N = (size_t)N;
  h->prec = (int)prec;
  if (bc) h->bc = *bc;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->params.theta = prec == ELBM_F64 ? 1e-8 : 3e-4;
  h->params.eps = 0.0;
  h->params.fallback = 1;
  cudaError_t e = cudaGetDevice(&h->device);
  const size_t pb = 27 * h->N * elem_size(h->prec);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMalloc(&h->pops[b], pb);
    if (e == cudaSuccess && is_dev_format(h->prec)) e = cudaMalloc((void**)&h->scale[b], h->N * sizeof(float));
  }
  StateIO S = state_io(h);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_counters, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_scratch, reduce_blocks(S) * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_out4, 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_counters, 0, 8 * sizeof(unsigned long long), h->stream);
  if (e != cudaSuccess) {
    elbm_status s = e == cudaErrorMemoryAllocation ? ELBM_ERR_OOM : ELBM_ERR_CUDA;
    elbm_destroy(h);
    return s;
  }
  rebuild_consts(h);
  *out = h;
  return ELBM_OK;
}

void elbm_destroy(elbm_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (int b = 0; b < 2; ++b) {
    cudaFree(h->pops[b]);
    cudaFree(h->scale[b]);
  }
  cudaFree(h->T6);
  cudaFree(h->src);
  cudaFree(h->u3);
  cudaFree(h->d_counters);
  cudaFree(h->d_scratch);
  cudaFree(h->d_out4);
  delete h;
}

const char* elbm_last_error(elbm_handle h) { return h ? h->err.c_str() : "null handle"; }

elbm_status elbm_set_params(elbm_handle h, const elbm_params* p) {
  if (!h || !p) return fail(h, ELBM_ERR_ARG, "null argument");
  if (!(p->theta >= 0.0) || !std::isfinite(p->eps)) return fail(h, ELBM_ERR_ARG, "theta must be >= 0, eps finite");
  h->params = *p;
  rebuild_consts(h);
  return ELBM_OK;
}

elbm_status elbm_set_tensor_uniform(elbm_handle h, const double D6[6]) {
  if (!h || !D6) return fail(h, ELBM_ERR_ARG, "null argument");
  if (!spd6(D6)) return fail(h, ELBM_ERR_NOT_SPD, "tensor is not symmetric positive definite");
  std::memcpy(h->D6, D6, sizeof(h->D6));
  h->have_tensor = true;
  h->tensor_field = false;
  rebuild_consts(h);
  return ELBM_OK;
}

static elbm_status set_field(elbm_handle h, const float* in, int is_params) {
  if (!h || !in) return fail(h, ELBM_ERR_ARG, "null argument");
  const size_t tb = h->prec == 0 ? sizeof(double) : sizeof(float);
  if (!h->T6) CK(cudaMalloc(&h->T6, 6 * h->N * tb), "cudaMalloc T6");
  const void* dev;
  void* tmp;
  elbm_status s = to_device(h, in, 6 * h->N * sizeof(float), &dev, &tmp);
  if (s != ELBM_OK) return s;
  CK(cudaMemsetAsync(h->d_counters + 1, 0, sizeof(unsigned long long), h->stream), "memset");
  CK(launch_tensor_prepass(static_cast<const float*>(dev), is_params, h->T6, h->prec == 0, h->N, h->d_counters + 1,
                           h->stream),
     "tensor pre-pass");
  unsigned long long bad = 0;
  CK(cudaMemcpyAsync(&bad, h->d_counters + 1, sizeof(bad), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  if (tmp) cudaFreeAsync(tmp, h->stream);
  CK(cudaStreamSynchronize(h->stream), "sync");
  if (bad) {
    h->have_tensor = false;
    return fail(h, ELBM_ERR_NOT_SPD, std::to_string(bad) + " nodes with a non-SPD or non-finite tensor");
  }
  h->have_tensor = true;
  h->tensor_field = true;
  rebuild_consts(h);
  return ELBM_OK;
}

elbm_status elbm_set_tensor_field(elbm_handle h, const float* D6) { return set_field(h, D6, 0); }
elbm_status elbm_set_tensor_params_field(elbm_handle h, const float* theta6) { return set_field(h, theta6, 1); }

elbm_status elbm_set_velocity_uniform(elbm_handle h, const double u[3]) {
  if (!h || !u) return fail(h, ELBM_ERR_ARG, "null argument");
  if (elbm_check_velocity(u) != ELBM_OK) return fail(h, ELBM_ERR_MACH, "velocity gives a non-positive P_i(u)");
  if (h->initialized) return fail(h, ELBM_ERR_STATE, "velocity must be set before the state is initialised");
  std::memcpy(h->u, u, sizeof(h->u));
  if (h->u3) {
    CK(cudaStreamSynchronize(h->stream), "sync");
    cudaFree(h->u3);
    h->u3 = nullptr;
  }
  rebuild_consts(h);
  return ELBM_OK;
}

elbm_status elbm_set_velocity_field(elbm_handle h, const float* u3) {
  if (!h || !u3) return fail(h, ELBM_ERR_ARG, "null argument");
  if (h->initialized) return fail(h, ELBM_ERR_STATE, "velocity must be set before the state is initialised");
  if (!h->u3) CK(cudaMalloc((void**)&h->u3, 3 * h->N * sizeof(float)), "cudaMalloc velocity field");
  CK(cudaMemcpyAsync(h->u3, u3, 3 * h->N * sizeof(float), cudaMemcpyDefault, h->stream), "memcpy velocity");
  CK(cudaMemsetAsync(h->d_counters + 1, 0, sizeof(unsigned long long), h->stream), "memset");
  CK(launch_velocity_check(h->u3, h->N, h->d_counters + 1, h->stream), "velocity check");
  unsigned long long bad = 0;
  CK(cudaMemcpyAsync(&bad, h->d_counters + 1, sizeof(bad), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  CK(cudaStreamSynchronize(h->stream), "sync");
  if (bad) {
    cudaFree(h->u3);
    h->u3 = nullptr;
    return fail(h, ELBM_ERR_MACH, std::to_string(bad) + " nodes whose velocity gives a non-positive P_i(u)");
  }
  // the deviation storages encode relative to the zero-velocity equilibrium shape
  h->u[0] = h->u[1] = h->u[2] = 0.0;
  rebuild_consts(h);
  return ELBM_OK;
}

elbm_status elbm_set_source(elbm_handle h, const float* R) {
  if (!h) return ELBM_ERR_ARG;
  if (h->initialized) return fail(h, ELBM_ERR_STATE, "source must be set before the state is initialised");
  if (!R) {
    CK(cudaStreamSynchronize(h->stream), "sync");
    cudaFree(h->src);
    h->src = nullptr;
    return ELBM_OK;
  }
  if (!h->src) CK(cudaMalloc((void**)&h->src, h->N * sizeof(float)), "cudaMalloc source");
  CK(cudaMemcpyAsync(h->src, R, h->N * sizeof(float), cudaMemcpyDefault, h->stream), "memcpy source");
  return ELBM_OK;
}

static elbm_status write_state(elbm_handle h, const void* in, elbm_dtype dt, int from_phi) {
  if (!h || !in) return fail(h, ELBM_ERR_ARG, "null argument");
  if (dt != ELBM_DTYPE_F64 && dt != ELBM_DTYPE_F32) return fail(h, ELBM_ERR_ARG, "bad dtype");
  const size_t bytes = (from_phi ? 1 : 27) * h->N * (dt == ELBM_DTYPE_F64 ? 8 : 4);
  const void* dev;
  void* tmp;
  elbm_status s = to_device(h, in, bytes, &dev, &tmp);
  if (s != ELBM_OK) return s;
  StateIO S = state_io(h);
  CK(launch_write_state(S, dev, dt == ELBM_DTYPE_F32, from_phi, h->stream), "write state");
  if (tmp) CK(cudaFreeAsync(tmp, h->stream), "cudaFreeAsync");
  CK(cudaMemsetAsync(h->d_counters, 0, sizeof(unsigned long long), h->stream), "memset");
  CK(cudaMemsetAsync(h->d_counters + 3, 0, sizeof(unsigned long long), h->stream), "memset");
  h->step = 0;
  h->initialized = true;
  return ELBM_OK;
}

elbm_status elbm_init_equilibrium(elbm_handle h, const void* phi0, elbm_dtype dt) {
  return write_state(h, phi0, dt, 1);
}

elbm_status elbm_write_populations(elbm_handle h, const void* g, elbm_dtype dt) { return write_state(h, g, dt, 0); }

static elbm_status read_state(elbm_handle h, void* out, void* q, elbm_dtype dt, int what) {
  if (!h || !out) return fail(h, ELBM_ERR_ARG, "null argument");
  if (!h->initialized) return fail(h, ELBM_ERR_STATE, "state not initialised");
  if (dt != ELBM_DTYPE_F64 && dt != ELBM_DTYPE_F32) return fail(h, ELBM_ERR_ARG, "bad dtype");
  const size_t es = dt == ELBM_DTYPE_F64 ? 8 : 4;
  const size_t b1 = (what == 0 ? 27 : 1) * h->N * es, bq = 3 * h->N * es;
  const bool host = !is_device_ptr(out);
  const bool qhost = q && !is_device_ptr(q);
  void* dout = out;
  void* dq = q;
  if (host) CK(cudaMallocAsync(&dout, b1, h->stream), "cudaMallocAsync");
  if (qhost) CK(cudaMallocAsync(&dq, bq, h->stream), "cudaMallocAsync");
  StateIO S = state_io(h);
  CK(launch_read_state(S, dout, dq, dt == ELBM_DTYPE_F32, what, h->stream), "read state");
  if (host) {
    CK(cudaMemcpyAsync(out, dout, b1, cudaMemcpyDeviceToHost, h->stream), "memcpy D2H");
    CK(cudaFreeAsync(dout, h->stream), "free");
  }
  if (qhost) {
    CK(cudaMemcpyAsync(q, dq, bq, cudaMemcpyDeviceToHost, h->stream), "memcpy D2H");
    CK(cudaFreeAsync(dq, h->stream), "free");
  }
  if (host || qhost) CK(cudaStreamSynchronize(h->stream), "sync");
  return ELBM_OK;
}

elbm_status elbm_read_populations(elbm_handle h, void* out, elbm_dtype dt) { return read_state(h, out, nullptr, dt, 0); }

elbm_status elbm_read_moments(elbm_handle h, void* phi, void* q, elbm_dtype dt) { return read_state(h, phi, q, dt, 1); }

elbm_status elbm_step(elbm_handle h, int64_t nsteps) {
  if (!h) return ELBM_ERR_ARG;
  if (nsteps < 0) return fail(h, ELBM_ERR_ARG, "nsteps < 0");
  if (!h->initialized) return fail(h, ELBM_ERR_STATE, "state not initialised");
  if (!h->have_tensor) return fail(h, ELBM_ERR_STATE, "no diffusion tensor set");
  if (h->u3 && h->src)
    return fail(h, ELBM_ERR_UNSUPPORTED, "a source with a per-node velocity field is not supported");
  StepLaunch L;
  L.prec = h->prec;
  L.vel = h->u3 ? 2 : ((h->u[0] != 0.0 || h->u[1] != 0.0 || h->u[2] != 0.0) ? 1 : 0);
  L.u3 = h->u3;
  L.nx = h->nx;
  L.ny = h->ny;
  L.nz = h->nz;
  L.N = h->N;
  L.dirichlet = h->bc.dirichlet_x;
  L.fallback = h->params.fallback;
  L.T6 = h->tensor_field ? h->T6 : nullptr;
  L.src = h->src;
  L.counters = h->d_counters;
  L.kd = &h->kd;
  L.kf = &h->kf;
  L.variant = h->step_kernel;
  L.wait_limit = h->wait_limit;
  L.withheld = h->wait_withheld;
  for (int64_t s = 0; s < nsteps; ++s) {
    L.pin = h->pops[h->cur];
    L.sin = h->scale[h->cur];
    L.pout = h->pops[1 - h->cur];
    L.sout = h->scale[1 - h->cur];
    CK(launch_step(L, h->stream), "step kernel");
    h->cur = 1 - h->cur;
    h->step += 1;
  }
  return ELBM_OK;
}

elbm_status elbm_set_lambda_mode(elbm_handle h, int32_t mode) {
  if (!h || (mode != 0 && mode != 1)) return fail(h, ELBM_ERR_ARG, "mode must be 0 or 1");
  h->lambda_mode = mode;
  rebuild_consts(h);
  return ELBM_OK;
}

elbm_status elbm_set_step_kernel(elbm_handle h, int32_t variant) {
  if (!h || variant < 0 || variant > 3) return fail(h, ELBM_ERR_ARG, "variant must be 0, 1, 2 or 3");
  if (variant == 2 && !rows_eligible(h->prec, h->nx))
    return fail(h, ELBM_ERR_UNSUPPORTED, "staged-row step needs nx % 8 == 0 and rows that fit in shared memory");
  if (variant == 3) {
    const int vel = h->u3 ? 2 : ((h->u[0] != 0.0 || h->u[1] != 0.0 || h->u[2] != 0.0) ? 1 : 0);
    if (!pipe_eligible(h->prec, h->nx, vel, h->lambda_mode != 0))
      return fail(h, ELBM_ERR_UNSUPPORTED, "pipelined staged-row step needs nx % 8 == 0 and three row stages "
                                           "in shared memory");
  }
  h->step_kernel = variant;
  return ELBM_OK;
}

elbm_status elbm_set_wait_limit(elbm_handle h, int64_t cycles) {
  if (!h || cycles < 0) return fail(h, ELBM_ERR_ARG, "cycles must be >= 0");
  h->wait_limit = cycles;
  return ELBM_OK;
}

elbm_status elbm_set_wait_test(elbm_handle h, int32_t withheld) {
  if (!h || withheld < 0 || withheld > 8) return fail(h, ELBM_ERR_ARG, "withheld must be in [0, 8]");
  h->wait_withheld = withheld;
  return ELBM_OK;
}

elbm_status elbm_set_exact_mass(elbm_handle h, int32_t on) {
  if (!h || (on != 0 && on != 1)) return fail(h, ELBM_ERR_ARG, "on must be 0 or 1");
  h->exact_mass = on;
  rebuild_consts(h);
  return ELBM_OK;
}

elbm_status elbm_get_step_kernel(elbm_handle h, int32_t* variant) {
  if (!h || !variant) return fail(h, ELBM_ERR_ARG, "null argument");
  const int vel = h->u3 ? 2 : ((h->u[0] != 0.0 || h->u[1] != 0.0 || h->u[2] != 0.0) ? 1 : 0);
  *variant = step_variant(h->prec, h->nx, vel, h->lambda_mode != 0, h->step_kernel);
  return ELBM_OK;
}

// A staging wait of the step kernel gave up (counters[2]); clears the flag.
static elbm_status check_timeout(elbm_ctx* h) {
  unsigned long long t = 0;
  CK(cudaMemcpyAsync(&t, h->d_counters + 2, sizeof(t), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  CK(cudaStreamSynchronize(h->stream), "sync");
  if (t != 0) {
    CK(cudaMemsetAsync(h->d_counters + 2, 0, sizeof(t), h->stream), "memset");
    return fail(h, ELBM_ERR_TIMEOUT, "a staging wait in the step kernel ran out");
  }
  return ELBM_OK;
}

elbm_status elbm_set_source_amplitude(elbm_handle h, double a) {
  if (!h || !std::isfinite(a)) return fail(h, ELBM_ERR_ARG, "bad amplitude");
  if (h->initialized) return fail(h, ELBM_ERR_STATE, "the amplitude must be set before the state is initialised");
  h->src_amp = a;
  rebuild_consts(h);
  return ELBM_OK;
}

elbm_status elbm_step_source_schedule(elbm_handle h, const double* amp, int64_t nsteps) {
  if (!h || (nsteps > 0 && !amp)) return fail(h, ELBM_ERR_ARG, "null argument");
  if (nsteps < 0) return fail(h, ELBM_ERR_ARG, "nsteps < 0");
  for (int64_t s = 0; s < nsteps; ++s) {
    if (!std::isfinite(amp[s])) return fail(h, ELBM_ERR_ARG, "non-finite amplitude");
    const double a_prev = h->src_amp;
    // this step applies the trailing half of the previous step and the leading half of this one
    h->kd.src_step = 0.5 * (a_prev + amp[s]);
    h->kf.src_step = (float)h->kd.src_step;
    elbm_status st = elbm_step(h, 1);
    h->src_amp = amp[s];
    if (st != ELBM_OK) {
      rebuild_consts(h);
      return st;
    }
  }
  rebuild_consts(h);
  return ELBM_OK;
}

elbm_status elbm_reduce(elbm_handle h, double* mass, double* entropy, double* gmin, int64_t* n_fallback) {
  if (!h) return ELBM_ERR_ARG;
  if (!h->initialized) return fail(h, ELBM_ERR_STATE, "state not initialised");
  StateIO S = state_io(h);
  CK(launch_reduce(S, h->d_scratch, h->d_out4, h->stream), "reduce");
  double o[4];
  unsigned long long fb = 0;
  CK(cudaMemcpyAsync(o, h->d_out4, sizeof(o), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  CK(cudaMemcpyAsync(&fb, h->d_counters, sizeof(fb), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  CK(cudaStreamSynchronize(h->stream), "sync");
  if (mass) *mass = o[0];
  if (entropy) *entropy = o[1];
  if (gmin) *gmin = o[2];
  if (n_fallback) *n_fallback = (int64_t)fb;
  if (check_timeout(h) != ELBM_OK) return ELBM_ERR_TIMEOUT;
  if (o[3] > 0) return fail(h, ELBM_ERR_NONFINITE, std::to_string((long long)o[3]) + " non-finite populations");
  return ELBM_OK;
}

elbm_status elbm_storage_projections(elbm_handle h, int64_t* n) {
  if (!h || !n) return fail(h, ELBM_ERR_ARG, "null argument");
  unsigned long long c = 0;
  CK(cudaMemcpyAsync(&c, h->d_counters + 3, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  CK(cudaStreamSynchronize(h->stream), "sync");
  *n = (int64_t)c;
  return ELBM_OK;
}

elbm_status elbm_get_step(elbm_handle h, int64_t* step) {
  if (!h || !step) return fail(h, ELBM_ERR_ARG, "null argument");
  *step = h->step;
  return ELBM_OK;
}

elbm_status elbm_synchronize(elbm_handle h) {
  if (!h) return ELBM_ERR_ARG;
  CK(cudaStreamSynchronize(h->stream), "sync");
  CK(cudaGetLastError(), "async error");
  return check_timeout(h);
}

static size_t ckpt_bytes(elbm_ctx* h) {
  return 32 + 27 * h->N * elem_size(h->prec) + (is_dev_format(h->prec) ? h->N * sizeof(float) : 0);
}

elbm_status elbm_checkpoint_size(elbm_handle h, size_t* bytes) {
  if (!h || !bytes) return fail(h, ELBM_ERR_ARG, "null argument");
  *bytes = ckpt_bytes(h);
  return ELBM_OK;
}

elbm_status elbm_checkpoint_save(elbm_handle h, void* buf, size_t bytes) {
  if (!h || !buf) return fail(h, ELBM_ERR_ARG, "null argument");
  if (bytes < ckpt_bytes(h)) return fail(h, ELBM_ERR_ARG, "checkpoint buffer too small");
  if (!h->initialized) return fail(h, ELBM_ERR_STATE, "state not initialised");
  unsigned long long fb = 0;
  CK(cudaMemcpyAsync(&fb, h->d_counters, sizeof(fb), cudaMemcpyDeviceToHost, h->stream), "memcpy");
  CK(cudaStreamSynchronize(h->stream), "sync");
  int64_t hdr[4] = {0x454c424dll, h->step, (int64_t)fb, (int64_t)h->prec};
  char* b = static_cast<char*>(buf);
  CK(cudaMemcpyAsync(b, hdr, sizeof(hdr), cudaMemcpyDefault, h->stream), "memcpy");
  const size_t pb = 27 * h->N * elem_size(h->prec);
  CK(cudaMemcpyAsync(b + 32, h->pops[h->cur], pb, cudaMemcpyDefault, h->stream), "memcpy");
  if (is_dev_format(h->prec))
    CK(cudaMemcpyAsync(b + 32 + pb, h->scale[h->cur], h->N * sizeof(float), cudaMemcpyDefault, h->stream), "memcpy");
  CK(cudaStreamSynchronize(h->stream), "sync");
  return ELBM_OK;
}

elbm_status elbm_checkpoint_load(elbm_handle h, const void* buf, size_t bytes) {
  if (!h || !buf) return fail(h, ELBM_ERR_ARG, "null argument");
  if (bytes < ckpt_bytes(h)) return fail(h, ELBM_ERR_ARG, "checkpoint buffer too small");
  int64_t hdr[4];
  const char* b = static_cast<const char*>(buf);
  CK(cudaMemcpyAsync(hdr, b, sizeof(hdr), cudaMemcpyDefault, h->stream), "memcpy");
  CK(cudaStreamSynchronize(h->stream), "sync");
  if (hdr[0] != 0x454c424dll || hdr[3] != h->prec) return fail(h, ELBM_ERR_ARG, "not a checkpoint of this precision");
  const size_t pb = 27 * h->N * elem_size(h->prec);
  CK(cudaMemcpyAsync(h->pops[h->cur], b + 32, pb, cudaMemcpyDefault, h->stream), "memcpy");
  if (is_dev_format(h->prec))
    CK(cudaMemcpyAsync(h->scale[h->cur], b + 32 + pb, h->N * sizeof(float), cudaMemcpyDefault, h->stream), "memcpy");
  unsigned long long fb = (unsigned long long)hdr[2];
  CK(cudaMemcpyAsync(h->d_counters, &fb, sizeof(fb), cudaMemcpyHostToDevice, h->stream), "memcpy");
  CK(cudaStreamSynchronize(h->stream), "sync");
  h->step = hdr[1];
  h->initialized = true;
  return ELBM_OK;
}

elbm_status elbm_state_pointers(elbm_handle h, void** pops, void** scale) {
  if (!h) return ELBM_ERR_ARG;
  if (pops) *pops = h->pops[h->cur];
  if (scale) *scale = h->scale[h->cur];
  return ELBM_OK;
}

}  // extern "C"
