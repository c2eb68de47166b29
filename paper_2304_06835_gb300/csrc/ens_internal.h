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
  float abstol_f, reltol_f, dt0_f;  // FP32 copies (an FP32 solve never converts in its loop)
  int refill_min;   // persistent schedule: refill a warp's idle lanes once this many are idle
  unsigned long long seed;
  long long index_offset;
  unsigned long long* queue;  // persistent-schedule counter (device), zeroed before launch
  const int* order;           // persistent schedule: queue slot -> trajectory index (or null)
  double saveat[ENS_MAX_SAVE];
};

struct CostScratch {
  unsigned short* bucket;  // [N]
  unsigned int* hist;      // [kCostBuckets] bucket totals, then cursors
  int blocks;              // G <= kCostBlocks
  long long chunk;         // trajectories per block
};

struct LaunchCfg {
  int schedule;  // ENS_SCHED_DIRECT or ENS_SCHED_PERSISTENT (resolved)
  int block;
  int tpt;
  int num_sms;
};

// Launch one solve; returns the CUDA error of the launch.  Implemented per (precision, model)
// in the solve_<precision>_<model>.cu units.
cudaError_t launch_solve(int rhs_id, int alg, int dtype, const SolveArgs& a,
                         const LaunchCfg& cfg, cudaStream_t stream, bool* supported);

// Longest-expected-first ordering for the persistent schedule: fills order[0..N) with the
// trajectory indices sorted by decreasing cost key (counting sort over kCostBuckets
// log-spaced buckets).  bucket: [N] scratch, hist: [kCostBuckets] scratch.
constexpr int kCostBuckets = 1024;
constexpr int kCostBlocks = 256;
cudaError_t launch_cost_order(int rhs_id, int alg, int dtype, const SolveArgs& a,
                              unsigned short* bucket, unsigned int* hist, int* order,
                              cudaStream_t stream);

// Register / shared-memory attributes of the kernel a launch would use (for tuning).
cudaError_t solve_kernel_attrs(int rhs_id, int alg, int dtype, const LaunchCfg& cfg,
                               cudaFuncAttributes* attr, int* blocks_per_sm);

cudaError_t launch_philox(unsigned long long seed, long long index_offset, long long n_traj,
                          long long n_calls, unsigned int* out, cudaStream_t s);
cudaError_t launch_normals(unsigned long long seed, long long index_offset, long long n_traj,
                           long long n_per, int dtype, void* out, cudaStream_t s);

}  // namespace ens
