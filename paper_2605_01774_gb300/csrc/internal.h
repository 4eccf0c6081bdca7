// Launch interfaces between the C ABI (api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "collide.cuh"

namespace elbm {

struct StepLaunch {
  int prec;                     // elbm_precision
  int vel;                      // 0: u = 0, 1: uniform u, 2: per-node u field
  const float* u3;              // per-node velocity [3][N] (vel = 2), else null
  int nx, ny, nz;
  size_t N;
  int dirichlet, fallback;
  const void* pin;              // post-collision populations (storage elements)
  const float* sin;             // deviation scale plane in
  void* pout;
  float* sout;
  const void* T6;               // per-node T = 2I - S [6][N] (double for FP64, else float) or null
  const float* src;             // per-node source [N] or null
  unsigned long long* counters; // [0] fallback count, [2] staging wait ran out, [3] nodes stored
                                // as their equilibrium shape, [4..5] row tickets
  const PopConsts<double>* kd;  // host copies, passed by value to the kernel
  const PopConsts<float>* kf;
  int variant;                  // 0 auto, 1 one thread per node with global gathers, 2 staged rows,
                                // 3 staged rows with a producer warp and per-stage full/empty barriers
  long long wait_limit;         // staging waits of variants 2 and 3 give up after this many cycles
  int withheld;                 // variant 2, test hook: arrivals its stage barriers never get
};
cudaError_t launch_step(const StepLaunch& L, cudaStream_t s);
// The implementation launch_step runs (1 per-node, 2 staged rows) for a requested variant
// (0 = auto).
int step_variant(int prec, int nx, int vel, bool root, int requested);
// Staged-row kernel (step_rows.cu): usable when rows_eligible(prec, nx); else cudaErrorNotSupported.
bool rows_eligible(int prec, int nx);
cudaError_t launch_step_rows(const StepLaunch& L, cudaStream_t s);
// Pipelined staged-row kernel (step_rows.cu): usable when pipe_eligible(...).
bool pipe_eligible(int prec, int nx, int vel, bool root);
cudaError_t launch_step_pipe(const StepLaunch& L, cudaStream_t s);

// State transfer.  mode 0: populations [27][N] <-> caller; mode 1: phi0 [N] -> equilibrium.
struct StateIO {
  int prec, nx, ny, nz;
  size_t N;
  int dirichlet;
  void* pops;                   // storage buffer (read: const)
  float* scale;
  const void* T6;               // double for FP64, else float
  const float* u3;              // per-node velocity [3][N] or null
  const float* src;
  const PopConsts<double>* kd;
  const PopConsts<float>* kf;
};
cudaError_t launch_write_state(const StateIO& S, const void* in, int in_f32, int from_phi, cudaStream_t s);
// what: 0 = populations [27][N]; 1 = phi [N] and optional q [3][N]
cudaError_t launch_read_state(const StateIO& S, void* out, void* q_out, int out_f32, int what, cudaStream_t s);
// partials: scratch of >= reduce_blocks(N) * 4 doubles; out4: device (mass, entropy, gmin, nonfinite count)
size_t reduce_blocks(const StateIO& S);
cudaError_t launch_reduce(const StateIO& S, double* scratch, double* out4, cudaStream_t s);

// Count nodes of a [3][N] velocity field with some P_i(u) <= 0 or a non-finite component.
cudaError_t launch_velocity_check(const float* u3, size_t N, unsigned long long* bad, cudaStream_t s);

// Tensor pre-pass: D6 or theta6 (float [6][N]) -> T6 ([6][N], double if t6_f64 else float);
// bad_count counts non-SPD nodes.
cudaError_t launch_tensor_prepass(const float* in, int is_params, void* T6, int t6_f64, size_t N,
                                  unsigned long long* bad_count, cudaStream_t s);

}  // namespace elbm
