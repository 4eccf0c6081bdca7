/*
 * elbm_adjoint.h -- gradients of a concentration misfit with respect to per-node
 * tensor parameters, by a hand-written adjoint of the collide-stream step.
 *
 * Parameters per node, theta [6][N]: ln d1, ln d2, ln d3 (principal diffusivities)
 * and ZYZ Euler angles a, b, c; D = R diag(d) R^T with R = Rz(a) Ry(b) Rz(c)
 * (Sections 2.3 and 3.1), S = (I/2 + D/cs2)^-1 (Eq. method-s-from-d).  Periodic
 * lattice, uniform velocity u, initial state g = g_eq(phi0, u), steps of
 * Section 2.7 with the entropic amplitude of Eq. method-lambda (guard theta) and
 * the positivity fallback of Eq. method-alpha (which must stay inactive for the
 * gradient to be that of the smooth branch: its count is returned).
 *
 * Misfit: J = 1/2 sum_{t in obs} sum_x (phi_t(x) - phi*_t(x))^2 with phi_t the
 * zeroth moment after t steps.  The gradient is computed by a reverse sweep over
 * checkpoints taken every K steps, recomputing each K-step segment forward.
 *
 * Arrays are device pointers in the handle's precision (double for ELBM_F64,
 * float for ELBM_F32), layout [component][N] with node n = x + Nx (y + Ny z).
 */
#ifndef ELBM_ADJOINT_H
#define ELBM_ADJOINT_H

#include <stdint.h>

#include "elbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct elbm_adjoint_ctx* elbm_adjoint_handle;

/* Lattice dims[3] (each 1..4096, 27 N < 2^31), precision ELBM_F64 or ELBM_F32
 * (else ELBM_ERR_UNSUPPORTED).  Defaults: u = 0, theta = 1e-8, K = 50. */
elbm_status elbm_adjoint_create(const int64_t dims[3], elbm_precision prec, void* cuda_stream,
                                elbm_adjoint_handle* out);
void elbm_adjoint_destroy(elbm_adjoint_handle h);
const char* elbm_adjoint_last_error(elbm_adjoint_handle h);

/* Velocity (ELBM_ERR_MACH unless all P_i(u) > 0), stabilizer guard theta >= 0,
 * checkpoint interval K >= 1. */
elbm_status elbm_adjoint_configure(elbm_adjoint_handle h, const double u[3], double theta, int32_t checkpoint_every);

/* J (host double) for nsteps steps from g_eq(phi0, u); nobs (1..16) observation
 * steps obs_steps[] in 1..nsteps with targets [nobs][N]; if grad6 != NULL also
 * dJ/dtheta [6][N].  n_fallback (host, may be NULL) = node collisions of the
 * forward sweep that took the positivity fallback.  Synchronous. */
elbm_status elbm_adjoint_misfit(elbm_adjoint_handle h, const void* theta6, const void* phi0, int64_t nsteps,
                                int32_t nobs, const int64_t* obs_steps, const void* targets, double* J, void* grad6,
                                int64_t* n_fallback);

/* One step on caller states (for tests and custom losses): from pre-collision
 * populations g [27][N], g_next (if not NULL) receives the populations after one
 * collide-stream step; if gbar != NULL it receives the vector-Jacobian product
 * (d g_next / d g)^T gbar_next and grad6 (if not NULL) the parameter part
 * (d g_next / d theta)^T gbar_next.  Synchronous. */
elbm_status elbm_adjoint_step(elbm_adjoint_handle h, const void* theta6, const void* g, const void* gbar_next,
                              void* g_next, void* gbar, void* grad6);

#ifdef __cplusplus
}
#endif

#endif /* ELBM_ADJOINT_H */
