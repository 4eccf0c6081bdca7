/*
 * elbm_batch.h -- many independent periodic lattices stepped together (an
 * orientation / anisotropy sweep of the anisotropic ADE entropic LBM).
 *
 * Each domain d is a periodic cube of edge n_d (1..256) with its own uniform
 * diffusion tensor D_d (S_d = (I/2 + D_d/cs2)^-1, Eq. method-s-from-d), zero
 * velocity (so the entropic amplitude is lambda = 1, Eq. method-lambda), FP32
 * populations and the step of Section 2.7 (flux relaxation, ghost damping,
 * positivity fallback of Eq. method-alpha, streaming of Eq. method-lbe).
 *
 * Layout: domains are concatenated; node (x, y, z) of domain d has index
 * off_d + x + n_d (y + n_d z) with off_d = sum_{e<d} n_e^3.  Per-node caller
 * arrays (phi) use that concatenated order.  The library owns two population
 * buffers of 27 sum_d n_d^3 floats.
 *
 * Errors as in elbm.h; ELBM_ERR_TIMEOUT when a bounded device-side wait of the
 * persistent kernel ran out (reported by elbm_batch_synchronize).
 */
#ifndef ELBM_BATCH_H
#define ELBM_BATCH_H

#include <stdint.h>

#include "elbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct elbm_batch_ctx* elbm_batch_handle;

/* ndom domains with edges[ndom] and tensors D6[ndom][6] (xx, xy, xz, yy, yz, zz;
 * each SPD, else ELBM_ERR_NOT_SPD), work ordered on cuda_stream (NULL: the
 * library creates a stream that synchronises with the default stream; CUDA
 * graphs cannot be captured on the default stream). */
elbm_status elbm_batch_create(int32_t ndom, const int32_t* edges, const double* D6, void* cuda_stream,
                              elbm_batch_handle* out);
void elbm_batch_destroy(elbm_batch_handle h);
const char* elbm_batch_last_error(elbm_batch_handle h);

/* Total nodes, current tile (threads per block), resident blocks per SM of the
 * persistent kernel, and whether the last mode-0 run went through a CUDA graph
 * (1) or was launched directly because capture was refused (0); -1 before. */
elbm_status elbm_batch_info(elbm_batch_handle h, int64_t* total_nodes, int32_t* tile, int32_t* blocks_per_sm,
                            int32_t* persistent_in_graph);

/* Positivity threshold eps (Eq. method-alpha, default 0) and fallback on/off. */
elbm_status elbm_batch_set_params(elbm_batch_handle h, double eps, int32_t fallback);

/* Bound of the persistent kernel's grid-barrier wait in SM clock cycles (default
 * 2e9, about one second) and, for testing the timeout path, a number of extra
 * arrivals the barrier waits for (default 0; > 0 makes every wait run out). */
elbm_status elbm_batch_set_wait_limit(elbm_batch_handle h, int64_t cycles, int32_t extra_arrivals);

/* g = g_eq(phi0, 0) on every domain; phi0 is the concatenated [sum n^3] field,
 * FP32, host or device.  Resets the step and fallback counters and the error flag. */
elbm_status elbm_batch_init_equilibrium(elbm_batch_handle h, const float* phi0);

/* Advance every domain nsteps steps (asynchronous).
 *   mode 0: one persistent cooperative kernel for all steps (tiles taken round-robin,
 *           bounded grid barrier between steps), captured into a CUDA graph;
 *   mode 1: one batched launch per step over all tiles, the sequence captured into a graph;
 *   mode 2: one plain single-lattice launch per domain per step (reference path).
 * A graph is captured and instantiated on the first call with a given (mode, nsteps, state
 * buffer parity, block shape, eps, fallback, wait limit) and relaunched by later calls with
 * the same key (up to 8 kept per handle; the autotuner's shape changes discard them). */
elbm_status elbm_batch_step(elbm_batch_handle h, int64_t nsteps, int32_t mode);

/* Wait for the stream; ELBM_ERR_TIMEOUT if a barrier wait ran out. */
elbm_status elbm_batch_synchronize(elbm_batch_handle h);

/* Time `steps_per_trial` mode-0 steps for each candidate block shape (threads per
 * block 128 or 256, resident blocks per SM 1 .. occupancy) and keep the fastest.
 * The trials advance the state: re-initialise afterwards. */
elbm_status elbm_batch_autotune(elbm_batch_handle h, int32_t steps_per_trial, int32_t* tile_out,
                                int32_t* blocks_per_sm_out);

/* phi of every node (concatenated order), FP32, host or device. */
elbm_status elbm_batch_read_phi(elbm_batch_handle h, float* phi);

/* Pre-collision populations [27][n_d^3] of one domain, FP32, host or device. */
elbm_status elbm_batch_read_populations(elbm_batch_handle h, int32_t domain, float* out);

/* Node collisions that took the positivity fallback since the last init. */
elbm_status elbm_batch_fallback_count(elbm_batch_handle h, int64_t* n);

#ifdef __cplusplus
}
#endif

#endif /* ELBM_BATCH_H */
