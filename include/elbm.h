/*
 * elbm.h -- C ABI of the GB300 (sm_103a) implementation of the entropic lattice
 * Boltzmann method for the full-tensor anisotropic advection-diffusion equation
 * (arXiv 2605.01774).
 *
 * Lattice: D3Q27 tensor-product set, c_i in {-1,0,1}^3, i = 9(cx+1)+3(cy+1)+(cz+1),
 * W_i = (2/3)^(3-m_i) (1/6)^(m_i), cs^2 = 1/3, dx = dt = 1 (Section 2.1).
 *
 * One time step (Section 2.7): pull-stream, phi = sum g, j = sum c (g - g_eq),
 * split g - g_eq = P(j) + dh, relax the flux with S = (I/2 + D/cs2)^-1
 * (Eq. method-s-from-d), damp the ghost dh with the ADE-corrected entropic
 * amplitude lambda (Eqs. method-lambda, method-correction), shorten the whole
 * increment by the positivity fallback alpha (Eq. method-alpha), write back.
 *
 * Layout and ownership
 *   Node (x, y, z) has linear index n = x + Nx (y + Ny z); every per-node field
 *   is a plane of N = Nx Ny Nz values, vector fields are [k][N] (component
 *   planes).  The library owns the population buffers and all derived data; the
 *   caller owns every pointer it passes and keeps it alive only for the call.
 *   Arguments documented "host or device" may point to either; the library asks
 *   the CUDA runtime which one it is.  Device pointers must belong to the
 *   current device.
 *
 * Streams and errors
 *   Work is ordered on the stream given to elbm_create (NULL = legacy default
 *   stream).  Calls that return data to host memory synchronise that stream;
 *   elbm_step only enqueues.  Every call returns an elbm_status; there are no
 *   exceptions across the ABI.  elbm_last_error() gives a message for the last
 *   failing call on a handle.  Kernel-side problems (non-finite populations,
 *   a timed-out wait) are reported by the next synchronising call.
 *
 * Thread safety: a handle may be used by one host thread at a time.
 */
#ifndef ELBM_H
#define ELBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ELBM_OK = 0,
    ELBM_ERR_ARG = 1,          /* bad argument (null, size, dtype, sizes mismatch) */
    ELBM_ERR_NOT_SPD = 2,      /* diffusion tensor not symmetric positive definite */
    ELBM_ERR_MACH = 3,         /* velocity makes an equilibrium weight P_i(u) <= 0 */
    ELBM_ERR_OOM = 4,          /* device allocation failed */
    ELBM_ERR_CUDA = 5,         /* CUDA runtime error (message in elbm_last_error) */
    ELBM_ERR_NONFINITE = 6,    /* non-finite population detected by a reduction */
    ELBM_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up */
    ELBM_ERR_STATE = 8,        /* call not valid in the handle's state (e.g. no init) */
    ELBM_ERR_UNSUPPORTED = 9   /* combination not available in this precision */
} elbm_status;

/* Storage and arithmetic of the populations.
 *   ELBM_F64          FP64 storage, FP64 arithmetic.
 *   ELBM_F32          FP32 storage, FP32 arithmetic.
 *   ELBM_F32_F16DEV   FP32 arithmetic; per node one FP32 scale phi_s and 27 FP16
 *                     relative deviations q_i, g_i = W_i phi_s (P_i(u) + q_i).
 *   ELBM_F32_BF16DEV  as above with BF16 deviations.
 * Reductions (mass, entropy) always accumulate in FP64. */
typedef enum { ELBM_F64 = 0, ELBM_F32 = 1, ELBM_F32_F16DEV = 2, ELBM_F32_BF16DEV = 3 } elbm_precision;

/* Element type of caller arrays handed to read/write calls. */
typedef enum { ELBM_DTYPE_F64 = 0, ELBM_DTYPE_F32 = 1 } elbm_dtype;

/* Boundaries.  dirichlet_x = 0: periodic in x, y, z.  dirichlet_x = 1: x faces
 * held at phi_lo (wall at x = -1/2) and phi_hi (wall at x = Nx - 1/2) by
 * anti-bounce-back, g_i(x_b) = -g*_opp(i)(x_b) + 2 W_i phi_w (wall velocity 0);
 * y and z stay periodic.  (Section 4.2.1 names the faces but gives no scheme.) */
typedef struct {
    int32_t dirichlet_x;
    double phi_lo;
    double phi_hi;
} elbm_bc;

/* Run-time parameters (defaults in brackets).
 *   theta     stabilizer guard: lambda = 1 where <dh|dh>_H <= theta^2 phi
 *             [1e-8 for ELBM_F64, 3e-4 otherwise]; "if dh = 0 set lambda = 1",
 *             Eq. (method-lambda), given a threshold.
 *   eps       positivity threshold of Eq. (method-alpha) [0].
 *   fallback  1 = positivity fallback on [1]. */
typedef struct {
    double theta;
    double eps;
    int32_t fallback;
} elbm_params;

typedef struct elbm_ctx* elbm_handle;

/* ---------------------------------------------------------------- lifecycle */

/* Create a lattice of dims[0] x dims[1] x dims[2] = Nx x Ny x Nz nodes (each >= 1,
 * total 27 N < 2^31 per population buffer index space) in precision `prec`,
 * boundaries `bc` (NULL = fully periodic), work ordered on `cuda_stream`
 * (a cudaStream_t, NULL = default stream).  Allocates two population buffers
 * (A/B) on the current device.  Initial tensor: D = 0 is not allowed, so a
 * tensor must be set before the first step; velocity 0; no source.
 * Errors: ELBM_ERR_ARG, ELBM_ERR_OOM, ELBM_ERR_CUDA. */
elbm_status elbm_create(const int64_t dims[3], elbm_precision prec, const elbm_bc* bc,
                        void* cuda_stream, elbm_handle* out);

/* Free every device buffer of the handle (after synchronising its stream). */
void elbm_destroy(elbm_handle h);

/* Message of the last failing call on `h` ("" if none); valid until the next call. */
const char* elbm_last_error(elbm_handle h);

/* Name of a status code. */
const char* elbm_status_string(elbm_status s);

/* Set theta, eps, fallback (see elbm_params).  ELBM_ERR_ARG if theta < 0. */
elbm_status elbm_set_params(elbm_handle h, const elbm_params* p);

/* How the entropic amplitude lambda is obtained where the ghost content is above the
 * guard.  mode 0 (default): the closed form of Eqs. (method-lambda, method-correction),
 * which the paper uses in all its runs.  mode 1: the exact root of the entropy-
 * stationarity condition, Eq. (method-entropy-root), sum_i dh_i ln((g_eq_i + ds_post_i +
 * (1 - lambda) dh_i)/W_i) = 0, solved per node by safeguarded Newton in FP64 (for every
 * precision) from the closed-form value inside the bracket where all arguments are
 * positive; the closed form is kept where that bracket is empty.  Mode 1 is costly (27
 * FP64 logarithms per Newton iteration) and applies only where u != 0.
 * ELBM_ERR_ARG for other modes. */
elbm_status elbm_set_lambda_mode(elbm_handle h, int32_t mode);

/* Which implementation of the fused collide-stream step (Eq. method-lbe with the collision
 * of Eqs. method-split..method-fallback) elbm_step launches; all give the same result up to
 * the order of floating-point operations, which is identical (bit-equal outputs).
 *   0 (default) auto: 2 for the FP32-arithmetic storages where nx >= 256 (row lengths 256,
 *     384 and 512 compiled in) with a uniform velocity and the closed-form stabilizer
 *     (measured faster there), else 1 (rows shorter than a block, per-node velocity fields,
 *     the exact-root stabilizer and FP64 measured faster with 1).
 *   1 one thread per node gathering its 27 pulled populations from global memory.
 *   2 persistent blocks taking x-rows from a ticket counter and staging each row's 27
 *     pulled source rows (and, for the deviation storages, the 9 scale rows; with a tensor
 *     field or a source also the row's 6 T rows and source row where they fit) in shared
 *     memory with asynchronous bulk copies, two buffers deep; needs nx % 8 == 0 and the
 *     buffers within 200 KiB: nx <= 472 in FP64, 944 in FP32, 1136 in the deviation
 *     storages.
 *   3 no block barrier per row: persistent blocks (two per SM, one for FP64), each a producer
 *     warp feeding a ring of row stages (per-stage full/empty mbarriers) to consumer warps that
 *     take 32-node segments and release a stage once their populations are loaded; needs
 *     nx % 8 == 0 and at least three stages in shared memory.  Measured no faster than 2 on
 *     GB300 (the default never picks it).
 * ELBM_ERR_ARG for other values, ELBM_ERR_UNSUPPORTED for 2 or 3 where it is not available.
 * A bounded staging wait that gives up makes the next elbm_synchronize or elbm_reduce
 * return ELBM_ERR_TIMEOUT (see elbm_set_wait_limit). */
elbm_status elbm_set_step_kernel(elbm_handle h, int32_t variant);

/* Limit, in SM clock cycles, of every wait of the staged-row step kernels (variants 2 and 3)
 * for a row's copies or a stage's release; cycles = 0 restores the default (2e9, about one
 * second at 2 GHz).  A wait that runs out makes its block stop, wait (with the default limit)
 * for the copies it issued, and leave; the next elbm_synchronize or elbm_reduce returns
 * ELBM_ERR_TIMEOUT and the state is then undefined until the next elbm_init_* or
 * elbm_write_populations.  Limits below 2^20 cycles are checked with non-blocking probes of
 * the barrier (cycle-accurate); longer ones with blocking probes, which the hardware may
 * hold for a short time of its own.  Meant for detecting a stalled device without hanging
 * the host.
 * ELBM_ERR_ARG if cycles < 0. */
elbm_status elbm_set_wait_limit(elbm_handle h, int64_t cycles);

/* Test hook for the bounded staging waits of variant 2 (no counterpart in the paper): with
 * withheld = k > 0 every row-stage barrier of the staged-row kernel expects k more arrivals
 * than the kernel makes, so the first staging wait of every block runs out after the limit of
 * elbm_set_wait_limit.  The block then takes its abort path: the thread that issued the
 * copies makes the k missing arrivals itself and waits (bounded) until the copies in flight
 * have landed, and the next elbm_synchronize or elbm_reduce returns ELBM_ERR_TIMEOUT; the
 * state is undefined until the next elbm_init_* or elbm_write_populations.  withheld = 0
 * (the default) restores normal stepping.  Variants 1 and 3 ignore it.
 * ELBM_ERR_ARG unless 0 <= withheld <= 8. */
elbm_status elbm_set_wait_test(elbm_handle h, int32_t withheld);

/* FP32 storage only (no effect on the others): with on = 1 (the default) each node update
 * puts the rounding of its 27 post-collision values back on its rest population c = 0, so the
 * stored node mass equals the conserved phi of Eq. (method-collision) up to one FP32
 * summation (the deviation storages keep their mass exactly by construction, FP64 to its
 * rounding).  With on = 0 the rounding of the updates acts as a small correlated source: on
 * the 256^3 plume of Section 3.1 the total mass drifts by 7.5e-4 over 40 000 steps (1e-7 with
 * on = 1).  Costs 1 to 4 % of the FP32 step time (more where the collision, not HBM, sets the
 * pace).  ELBM_ERR_ARG unless on is 0 or 1. */
elbm_status elbm_set_exact_mass(elbm_handle h, int32_t on);

/* The implementation (1 or 2, as above) elbm_step launches with the handle's current
 * storage, size, velocity, stabilizer mode and elbm_set_step_kernel choice. */
elbm_status elbm_get_step_kernel(elbm_handle h, int32_t* variant);

/* --------------------------------------------------------- problem data */

/* Uniform tensor D, 6 doubles (Dxx, Dxy, Dxz, Dyy, Dyz, Dzz), host memory.
 * Derives S = (I/2 + 3 D)^-1 (Eq. method-s-from-d) in FP64 on the host and keeps
 * T = 2I - S = 12 D (I + 6 D)^-1, which holds weak-axis diffusivities to full
 * relative precision in FP32.  ELBM_ERR_NOT_SPD unless D is SPD. */
elbm_status elbm_set_tensor_uniform(elbm_handle h, const double D6[6]);

/* Per-node tensor, FP32 [6][N] in the same component order, host or device.
 * A device pre-pass converts it once to the per-node T field (FP32 [6][N],
 * kept by the library).  Nodes whose D is not SPD make the call fail with
 * ELBM_ERR_NOT_SPD (checked on the device). */
elbm_status elbm_set_tensor_field(elbm_handle h, const float* D6);

/* Per-node tensor from parameters theta, FP32 [6][N], host or device:
 * theta[0..2] = ln d1, ln d2, ln d3 (principal diffusivities), theta[3..5] =
 * ZYZ Euler angles (a, b, c) in radians, D = Rz(a) Ry(b) Rz(c) diag(d) R^T
 * (Sections 2.3 and 3.1).  Converted once to the T field on the device. */
elbm_status elbm_set_tensor_params_field(elbm_handle h, const float* theta6);

/* Uniform velocity u (3 doubles, host).  ELBM_ERR_MACH unless every
 * P_i(u) = 1 + 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u > 0.  The velocity is part of the
 * stored-state convention (deviation reference, source half-steps), so it may only
 * be changed before elbm_init_* (else ELBM_ERR_STATE). */
elbm_status elbm_set_velocity_uniform(elbm_handle h, const double u[3]);

/* Per-node velocity u(x), FP32 [3][N] (component planes), host or device, copied by
 * the library.  Every node collides with the equilibrium of its own velocity
 * (Eq. method-geq), j = sum c g - phi u(x), and the stabilizer tables P_i(u(x)),
 * ln P_i(u(x)) of Eqs. (method-lambda, method-correction) are evaluated per node
 * (lambda = 1 where u(x) = 0 exactly).  ELBM_ERR_MACH (field discarded) if some node
 * has a P_i(u) <= 0; only before elbm_init_* (ELBM_ERR_STATE).  The deviation storages
 * then encode relative to the zero-velocity shape.  A source together with a velocity
 * field is ELBM_ERR_UNSUPPORTED at elbm_step.  elbm_set_velocity_uniform removes it. */
elbm_status elbm_set_velocity_field(elbm_handle h, const float* u3);

/* Time-constant volumetric source R, FP32 [N], host or device, or NULL to
 * remove it.  Applied by the Strang split S(1/2) -> collide-stream -> S(1/2),
 * g_i += (1/2) R E_i(u) with E_i(u) = W_i P_i(u) (Section 3.3); the two
 * half-steps between consecutive steps are merged into one full step. */
elbm_status elbm_set_source(elbm_handle h, const float* R);

/* Amplitude a of the source for time-dependent sources R(x, t) = a(t) R(x) (Section
 * 3.3 evaluates R at the mid-step time t_{n+1/2} for both half-steps of step n).  Sets the
 * amplitude of the half-step the stored state is considered to include; must be called
 * before elbm_init_* (ELBM_ERR_STATE otherwise).  Default 1. */
elbm_status elbm_set_source_amplitude(elbm_handle h, double a);

/* Advance nsteps steps with source amplitudes amp[0..nsteps-1] (host), amp[k] = a(t_{n+1/2})
 * of step n = current step + k.  Step n adds (a_{n-1} + a_n)/2 R E_i to the pulled
 * populations (trailing half of step n-1 merged with the leading half of step n); reads
 * and writes of the state then include a_{n-1}/2 R E_i.  With a constant amplitude this
 * is elbm_step. */
elbm_status elbm_step_source_schedule(elbm_handle h, const double* amp, int64_t nsteps);

/* --------------------------------------------------------------- state */

/* Initial state g = g_eq(phi0, u) (initial populations are not stated in the
 * paper; the equilibrium start is this library's reading).  phi0 is [N] of
 * `dtype`, host or device.  Resets the step counter and the fallback count. */
elbm_status elbm_init_equilibrium(elbm_handle h, const void* phi0, elbm_dtype dtype);

/* Set the state from pre-collision populations g [27][N] of `dtype` (host or
 * device): the populations that the next step collides, after the trailing
 * source half-step of the previous step.  For the deviation storages the
 * values are rounded to the storage format. */
elbm_status elbm_write_populations(elbm_handle h, const void* g, elbm_dtype dtype);

/* Read the current pre-collision populations g [27][N] into `out` (host or
 * device) as `dtype`.  Synchronises the stream when `out` is host memory. */
elbm_status elbm_read_populations(elbm_handle h, void* out, elbm_dtype dtype);

/* Read phi = sum_i g_i [N] and, if q_out != NULL, the LB diffusive flux
 * q = j - S j / 2 [3][N] (Eq. app-cube-lb-flux) of the current state.
 * Buffers host or device of `dtype`. */
elbm_status elbm_read_moments(elbm_handle h, void* phi_out, void* q_out, elbm_dtype dtype);

/* Advance `nsteps` >= 0 collide-stream steps (asynchronous on the stream). */
elbm_status elbm_step(elbm_handle h, int64_t nsteps);

/* Conservation diagnostics of the current state, FP64 (host pointers, any may
 * be NULL): mass = sum_x phi, entropy = sum_x sum_i g_i ln(g_i/W_i) over
 * positive g_i (Eq. method-entropy), gmin = min g_i, n_fallback = node
 * collisions that took the positivity fallback since the last init.
 * Deterministic (fixed-order two-pass reduction).  Returns ELBM_ERR_NONFINITE
 * (values still written) if any population is NaN or infinite. */
elbm_status elbm_reduce(elbm_handle h, double* mass, double* entropy, double* gmin,
                        int64_t* n_fallback);

/* Deviation storages: node updates, since the last init, whose 16-bit deviations could not
 * hold the node's shape (saturation, or a net mass far below the populations' magnitudes,
 * detected as a mass correction sum_i 2^-e_i v_i of magnitude 1/2 or more) and that were
 * stored as their equilibrium shape with their mass kept.  Always 0 for FP64 and FP32. */
elbm_status elbm_storage_projections(elbm_handle h, int64_t* n);

/* Steps taken since the last init. */
elbm_status elbm_get_step(elbm_handle h, int64_t* step);

/* Wait for the handle's stream; report asynchronous CUDA errors. */
elbm_status elbm_synchronize(elbm_handle h);

/* Checkpoints: byte size of a snapshot (populations in storage format + step
 * counter + fallback count), save into / load from a caller buffer (host or
 * device) of at least that size.  A snapshot is only valid for a handle of the
 * same dims and precision. */
elbm_status elbm_checkpoint_size(elbm_handle h, size_t* bytes);
elbm_status elbm_checkpoint_save(elbm_handle h, void* buf, size_t bytes);
elbm_status elbm_checkpoint_load(elbm_handle h, const void* buf, size_t bytes);

/* Device pointers of the current population buffer and (deviation storages)
 * of its FP32 scale plane, for profiling and zero-copy inspection.  They change
 * after every step (A/B swap).  Owned by the library. */
elbm_status elbm_state_pointers(elbm_handle h, void** pops, void** scale);

/* ------------------------------------------------ allocation-free diagnostics */

/* The paper has no counterpart of this call; it is a service for callers.
 *
 * Same diagnostics as elbm_reduce (mass, entropy, min g; out4[3] = number of
 * non-finite populations) for a population state the caller holds, computed
 * without allocating any device memory.  For callers that cannot allocate at
 * that moment: a process whose device memory is fully reserved by another
 * allocator (a framework's caching allocator, a memory pool owning the GPU), or
 * a monitoring hook inside a time-stepping loop where an allocation that blocks
 * or fails is not acceptable (e.g. reporting after an out-of-memory error).
 *
 * pops/scale: post-collision buffer in this library's storage layout for `prec`
 * (device pointers, e.g. from elbm_state_pointers; scale only for the deviation
 * formats, else NULL).  dims, bc: as given to the handle that produced the state
 * (bc NULL = periodic).  u: the handle's uniform velocity; (0, 0, 0) for a handle
 * with a per-node velocity field (elbm_set_velocity_field), whose deviation
 * storages encode against the zero-velocity equilibrium shape.  source: NULL, or
 * the handle's FP32 source plane R on the device multiplied by the amplitude a of
 * the source half-step the stored state includes (1 unless the amplitude was
 * changed with elbm_set_source_amplitude or elbm_step_source_schedule, where it is
 * the amplitude of the last step taken).  out4: 4 doubles, host or device.  Work is
 * ordered on cuda_stream; a host out4 synchronises it.  pops, scale and source must
 * be device memory of the current device (ELBM_ERR_ARG otherwise, nothing launched).
 *
 * Scratch: a fixed device array of 4096 partial sums (131 104 bytes per GPU
 * that loads the library, held until the process exits); the kernel strides over
 * the lattice, so every lattice the library accepts fits.  Lattices beyond the
 * library's limit (an axis above 65535, or 27 N >= 2^31) are rejected with
 * ELBM_ERR_ARG.  The first call on a device looks up the array's device address
 * (once per device and context, with that device current; again after the context
 * was destroyed and re-created, e.g. by cudaDeviceReset); make that first call before
 * any stream capture.  Every call reuses the same array and leaves its contents
 * behind: calls that overlap on the GPU (other streams, other host threads on
 * the same device) race and must be serialised by the caller.
 * Errors: ELBM_ERR_ARG, ELBM_ERR_CUDA. */
elbm_status elbm_reduce_noalloc(const void* pops, const float* scale, const int64_t dims[3],
                                elbm_precision prec, const double u[3], const elbm_bc* bc,
                                const float* source, void* cuda_stream, double out4[4]);

/* ------------------------------------------------ host-only validation (no GPU) */

/* ELBM_OK if D6 is SPD, else ELBM_ERR_NOT_SPD. */
elbm_status elbm_check_tensor(const double D6[6]);

/* ELBM_OK if P_i(u) > 0 for all i, else ELBM_ERR_MACH. */
elbm_status elbm_check_velocity(const double u[3]);

/* T = 2I - S (6 doubles) of an SPD D6, computed in FP64 on the host. */
elbm_status elbm_relaxation_complement(const double D6[6], double T6_out[6]);

/* Measured fused multiply-add throughput of the CUDA cores of the current device, in
 * flop/s (an FMA counts 2), for precision ELBM_F64 or ELBM_F32: many independent FMA
 * chains per thread over several waves of blocks, best of five timed launches.  It is the
 * arithmetic roofline of the FP64 step, which FP64 FMA issue bounds on this part.  The
 * paper has no counterpart.  ELBM_ERR_ARG for other precisions or a null pointer,
 * ELBM_ERR_CUDA on a runtime error.  Takes a few milliseconds; synchronises. */
elbm_status elbm_fma_peak(int32_t precision, double* flops_per_s);

/* Measured rate of bulk asynchronous global -> shared copies (cp.async.bulk completing on an
 * mbarrier) on the current device: blocks_per_sm persistent 256-thread blocks per SM, in each
 * of which warp 0 issues the copies (copy_bytes each, 24 KiB per stage, two stages) of a 1 GiB
 * source.  Returns the bytes and the copies per second of the whole device, best of three
 * timed launches.  It shows how fast one warp issues such copies (with small copies and few
 * issuing warps the issue rate, not DRAM, bounds the bytes), which is why the staged-row step
 * spreads a row's copies over all warps.  The paper has no counterpart.  ELBM_ERR_ARG unless
 * copy_bytes is a multiple of 16 in [16, 24576] and 1 <= blocks_per_sm <= 4, ELBM_ERR_OOM if
 * the 1 GiB source cannot be allocated, ELBM_ERR_TIMEOUT if a copy wait ran out (about one
 * second), ELBM_ERR_CUDA on a runtime error.  Allocates and frees device memory; synchronises. */
elbm_status elbm_bulk_copy_rate(int32_t copy_bytes, int32_t blocks_per_sm, double* bytes_per_s,
                                double* copies_per_s);

#ifdef __cplusplus
}
#endif

#endif /* ELBM_H */
