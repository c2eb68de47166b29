// ens_internal.h -- host/device shared argument block and the launcher table of libens.so.
#pragma once

#include <cuda_runtime.h>

#include "../../include/ens.h"

namespace ens {

// Everything a solve kernel reads, passed by value as the kernel parameter.
struct SolveArgs {
  long long N;
  const void* params;
  const void* u0;
  const void* tspan;
  void* out;
  signed char* status;
  int* stats;
  int layout;
  int n_save;
  double dt, abstol, reltol, dt0;
  long long maxiters;
  int maxiters_i;   // the same cap as an int (validated <= 2e9)
  int refill_min;   // persistent schedule: refill a warp's idle lanes once this many are idle
  unsigned long long seed;
  long long index_offset;
  unsigned long long* queue;  // persistent-schedule counter (device), zeroed before launch
  double saveat[ENS_MAX_SAVE];
};

struct LaunchCfg {
  int schedule;  // ENS_SCHED_DIRECT or ENS_SCHED_PERSISTENT (resolved)
  int block;
  int tpt;
  int num_sms;
};

// Launch one solve; returns the CUDA error of the launch.  Implemented per precision in
// solve_f32.cu / solve_f64.cu.
cudaError_t launch_solve(int rhs_id, int alg, int dtype, const SolveArgs& a,
                         const LaunchCfg& cfg, cudaStream_t stream, bool* supported);

// Register / shared-memory attributes of the kernel a launch would use (for tuning).
cudaError_t solve_kernel_attrs(int rhs_id, int alg, int dtype, const LaunchCfg& cfg,
                               cudaFuncAttributes* attr, int* blocks_per_sm);

cudaError_t launch_philox(unsigned long long seed, long long index_offset, long long n_traj,
                          long long n_calls, unsigned int* out, cudaStream_t s);
cudaError_t launch_normals(unsigned long long seed, long long index_offset, long long n_traj,
                           long long n_per, int dtype, void* out, cudaStream_t s);

}  // namespace ens
