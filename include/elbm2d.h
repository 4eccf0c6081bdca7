/*
 * elbm2d.h -- C ABI of the two-dimensional form of the anisotropic ADE entropic lattice
 * Boltzmann method (arXiv 2605.01774) on the D2Q9 tensor-product set.
 *
 * Lattice (Section 2.1): c_i in {-1,0,1}^2, i = 3 (cx+1) + (cy+1), W_i = (2/3)^(2-m_i)
 * (1/6)^(m_i) = 4/9, 1/9, 1/36 for m_i = 0, 1, 2 non-zero components, cs^2 = 1/3,
 * dx = dt = 1.  One step is the same sequence as in three dimensions (Section 2.7):
 * pull-stream, phi = sum g, j = sum c (g - g_eq), flux relaxation through
 * S = (I/2 + D/cs2)^-1 (Eq. method-s-from-d; kept as T = 2I - S), entropic amplitude of
 * the ghost sector (Eqs. method-lambda, method-correction, guard theta), positivity
 * fallback (Eq. method-alpha).  Section 4.1 runs the method on D2Q9 with tensor and
 * velocity fields that vary across the domain; both may be uniform or per node here.
 * Boundaries: periodic in x and y.
 *
 * Layout: node (x, y) has index n = x + Nx y; populations [9][N]; per-node fields are
 * component planes: tensor [3][N] (Dxx, Dxy, Dyy), velocity [2][N] (ux, uy).  The library
 * owns the population buffers and derived fields; the caller owns every pointer it passes.
 * Arguments documented "host or device" may point to either (device pointers of the
 * current device).  Status codes, elbm_params and elbm_dtype are those of elbm.h.  Work is
 * ordered on the stream given at creation; calls that return data to host memory
 * synchronise it.  A handle may be used by one host thread at a time.
 */
#ifndef ELBM2D_H
#define ELBM2D_H

#include "elbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct elbm2d_ctx* elbm2d_handle;

/* Create an Nx x Ny = dims[0] x dims[1] periodic lattice (each >= 1, N < 2^31) with
 * ELBM_F64 or ELBM_F32 storage and arithmetic (ELBM_ERR_UNSUPPORTED for the deviation
 * storages).  Allocates two population buffers on the current device.  Defaults: no
 * tensor (one must be set before stepping), u = 0, theta 1e-8 (FP64) / 3e-4 (FP32),
 * eps 0, fallback on.  Errors: ELBM_ERR_ARG, ELBM_ERR_OOM, ELBM_ERR_CUDA. */
elbm_status elbm2d_create(const int64_t dims[2], elbm_precision prec, void* cuda_stream, elbm2d_handle* out);

/* Free the handle's device buffers (after synchronising its stream). */
void elbm2d_destroy(elbm2d_handle h);

/* Message of the last failing call on `h` ("" if none). */
const char* elbm2d_last_error(elbm2d_handle h);

/* theta, eps, fallback as in elbm_set_params.  ELBM_ERR_ARG if theta < 0 or eps is not finite. */
elbm_status elbm2d_set_params(elbm2d_handle h, const elbm_params* p);

/* Uniform tensor D = (Dxx, Dxy, Dyy), host.  T = 2I - S = 12 D (I + 6 D)^-1 is formed in
 * FP64 on the host.  ELBM_ERR_NOT_SPD unless D is symmetric positive definite. */
elbm_status elbm2d_set_tensor_uniform(elbm2d_handle h, const double D3[3]);

/* Per-node tensor, FP32 [3][N] (Dxx, Dxy, Dyy), host or device; converted once on the
 * device to the per-node T field.  ELBM_ERR_NOT_SPD (field discarded) if some node's D is
 * not SPD or not finite. */
elbm_status elbm2d_set_tensor_field(elbm2d_handle h, const float* D3);

/* Uniform velocity (2 doubles, host).  ELBM_ERR_MACH unless every
 * P_i(u) = 1 + 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u > 0.  Removes a velocity field.  Only
 * before elbm2d_init_* / elbm2d_write_populations (ELBM_ERR_STATE otherwise). */
elbm_status elbm2d_set_velocity_uniform(elbm2d_handle h, const double u[2]);

/* Per-node velocity, FP32 [2][N], host or device, copied.  Every node uses the equilibrium
 * and stabilizer tables of its own u (lambda = 1 where that u is exactly 0).  ELBM_ERR_MACH
 * (field discarded) if some node has a P_i(u) <= 0; ELBM_ERR_STATE after initialisation. */
elbm_status elbm2d_set_velocity_field(elbm2d_handle h, const float* u2);

/* g = g_eq(phi0, u) from phi0 [N] of `dtype`, host or device.  Resets the step counter and
 * the fallback count. */
elbm_status elbm2d_init_equilibrium(elbm2d_handle h, const void* phi0, elbm_dtype dtype);

/* Set the state from pre-collision populations [9][N] of `dtype`, host or device. */
elbm_status elbm2d_write_populations(elbm2d_handle h, const void* g, elbm_dtype dtype);

/* Read the pre-collision populations [9][N] as `dtype` into host or device memory. */
elbm_status elbm2d_read_populations(elbm2d_handle h, void* out, elbm_dtype dtype);

/* Read phi = sum_i g_i [N] as `dtype` into host or device memory. */
elbm_status elbm2d_read_moments(elbm2d_handle h, void* phi_out, elbm_dtype dtype);

/* Advance nsteps >= 0 steps (asynchronous on the stream). */
elbm_status elbm2d_step(elbm2d_handle h, int64_t nsteps);

/* FP64 diagnostics of the current state (host pointers, any may be NULL): mass sum phi,
 * entropy sum g ln(g/W) over positive g (Eq. method-entropy), min g, and the number of node
 * collisions that took the positivity fallback since the last init.  ELBM_ERR_NONFINITE
 * (values still written) if a population is NaN or infinite. */
elbm_status elbm2d_reduce(elbm2d_handle h, double* mass, double* entropy, double* gmin, int64_t* n_fallback);

/* Wait for the handle's stream and report asynchronous CUDA errors. */
elbm_status elbm2d_synchronize(elbm2d_handle h);

/* ELBM_OK if P_i(u) > 0 for every D2Q9 velocity, else ELBM_ERR_MACH (host only). */
elbm_status elbm2d_check_velocity(const double u[2]);

/* T = 2I - S (Txx, Txy, Tyy) of an SPD D3 in FP64 on the host (ELBM_ERR_NOT_SPD otherwise). */
elbm_status elbm2d_relaxation_complement(const double D3[3], double T3_out[3]);

#ifdef __cplusplus
}
#endif

#endif /* ELBM2D_H */
