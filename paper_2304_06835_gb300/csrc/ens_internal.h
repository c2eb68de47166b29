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
  int step_cap;     // adaptive: store every accepted step (capacity per trajectory), 0: no
  void* step_t;     // times of the stored steps (or null)
  int* step_n;      // accepted steps + 1 (or null)
  double dtmax;     // adaptive: largest step (+inf when the caller set none)
  float dtmax_f;
  int refill_min;   // persistent schedule: refill a warp's idle lanes once this many are idle
  int dense;        // adaptive Tsit5 with save times: dense output instead of cut steps
  unsigned long long seed;
  long long index_offset;
  unsigned long long* queue;  // persistent-schedule counter (device), zeroed before launch
  const int* order;           // persistent schedule: queue slot -> trajectory index (or null)
  const void* h0;             // with the order: each trajectory's starting step (T[N], by
                              // trajectory index), formed by the ordering pre-pass; or null
  unsigned long long* slots;  // persistent schedule: adds the lane slots its warps issue (loop
                              // iterations x 32 x trajectories per thread), or null
  double saveat[ENS_MAX_SAVE];
  float saveat_f[ENS_MAX_SAVE];  // FP32 copies (no double conversion on FP32 solves' path)
};

// Arguments of the discrete-adjoint kernels (fixed-step explicit RK, one thread per trajectory).
struct AdjArgs {
  long long N;
  const void* params;
  const void* u0;
  const void* tspan;
  int layout;
  double dt;
  long long max_steps;   // capacity: every trajectory's step count must be <= max_steps
  int K;                 // checkpoint interval (steps)
  void* out;             // forward: final state [N][D] (layout) or null
  void* ckpt;            // [C][D][N] checkpoints u_{cK}, C = ceil(max_steps / K)
  const void* grad_out;  // [N][D] (layout) dL/du(tf)
  void* grad_p;          // [N][P] (layout)
  void* grad_u0;         // [N][D] (layout)
  signed char* status;   // [N] or null
  void* seg;             // [K][S][D][N] stage inputs of one segment (S stages of the method)
};

// Discrete adjoint: which = 0 forward with checkpoints, 1 reverse pass.  alg is
// ENS_TSIT5_FIXED or ENS_RK4.  Implemented in adjoint.cu.
cudaError_t launch_adjoint(int which, int rhs_id, int alg, int dtype, const AdjArgs& a,
                           cudaStream_t stream, bool* supported);
int adjoint_stages(int alg);  // stages whose inputs the reverse pass stores (0: unsupported)

struct CostScratch {
  float* keys = nullptr;   // [N]: set to write the raw cost keys instead of the buckets
  void* h0 = nullptr;      // [N] of the solve's type: the starting steps the keys are formed
                           // from (adaptive methods without a given dt0), or null
  unsigned short* bucket;  // [N]
  unsigned int* hist;      // [kCostBuckets] bucket totals
  int blocks;              // the keys pass's grid (it strides over all trajectories)
};

struct LaunchCfg {
  int schedule = ENS_SCHED_DIRECT;  // ENS_SCHED_DIRECT or ENS_SCHED_PERSISTENT (resolved)
  int block = 128;
  int tpt = 1;
  int num_sms = 1;
  int bps = 0;   // persistent: resident blocks per SM; 0 = as many as fit; < 0: -bps/4 of that
};

// Launch one solve; returns the CUDA error of the launch.  Implemented per (precision, model)
// in the solve_<precision>_<model>.cu units.
cudaError_t launch_solve(int rhs_id, int alg, int dtype, const SolveArgs& a,
                         const LaunchCfg& cfg, cudaStream_t stream, bool* supported);

// Longest-expected-first ordering for the persistent schedule: fills order[0..N) with the
// trajectory indices sorted by decreasing cost key (counting sort over kCostBuckets
// log-spaced buckets), and zeroes the persistent queue counter.  bucket: [N] scratch, hist:
// [kCostHistWords] scratch (the bucket totals, then the buckets' fill cursors); h0: the
// starting steps kept for the solve, or null; sms: the device's multiprocessors.
constexpr int kCostBuckets = 1024;
constexpr int kCostHistWords = 2 * kCostBuckets;
constexpr int kCostBlocks = 256;  // blocks of the scatter pass (one range per block and bucket)
cudaError_t launch_cost_order(int rhs_id, int alg, int dtype, const SolveArgs& a,
                              unsigned short* bucket, unsigned int* hist, int* order,
                              void* h0, unsigned long long* queue, int sms,
                              cudaStream_t stream);
// The cost keys themselves: keys[i] = the expected steps of trajectory i (the key the
// longest-first order sorts by).
cudaError_t launch_cost_keys(int rhs_id, int alg, int dtype, const SolveArgs& a, float* keys,
                             cudaStream_t stream);

// Device scratch of one persistent solve: the queue counter, and for the longest-first order
// the permutation [N], bucket keys [N] and the kCostBuckets bucket cursors.
struct SolveScratch {
  unsigned long long* queue;
  int* order;               // null: index order
  unsigned short* bucket;
  unsigned int* hist;
  void* h0 = nullptr;       // [N] of the solve's type, or null: the ordering pre-pass keeps the
                            // starting steps here for the solve's initialisation
};

// Shared pieces of the solve entry points (abi.cu).
int validate_problem(int rhs_id, long long N, const void* params, const void* u0,
                     const void* tspan, const ens_opts* o, const void* out);
void fill_solve_args(SolveArgs* a, long long N, const void* params, const void* u0,
                     const void* tspan, const ens_opts* o, void* out, signed char* status,
                     int* stats);
bool uses_cost_order(const ens_opts* o, const LaunchCfg& cfg);
// the steps of a persistent solve before its kernel: longest-first ordering into sc.order (sets
// a->order) and the queue reset (sets a->queue)
cudaError_t prepare_solve(int rhs_id, const ens_opts* o, SolveArgs* a, const LaunchCfg& cfg,
                          const SolveScratch& sc, cudaStream_t s);
// enqueue one solve on stream s: [cost order], queue reset, integrator kernel
cudaError_t enqueue_solve(int rhs_id, const ens_opts* o, SolveArgs a, const LaunchCfg& cfg,
                          const SolveScratch& sc, cudaStream_t s, bool* supported);
// launch shape of a solve: explicit options, else the autotuner's cache, else the defaults
// (persistent 128 x 1 for adaptive methods, direct 128 for fixed-step ones)
LaunchCfg resolve_launch(int rhs_id, long long N, const ens_opts* o, int num_sms);
int set_last_error(int code, const char* msg);
// Autotuner (batch.cu): time the candidate launch shapes of one solve on its own inputs and
// remember the fastest for resolve_launch; synchronises the stream.
int tune_problem(int rhs_id, const ens_opts* o, const SolveArgs& a, const SolveScratch& sc,
                 int sms, cudaStream_t s, LaunchCfg* best, float* best_ms);

// Register / shared-memory attributes of the kernel a launch would use (for tuning).
cudaError_t solve_kernel_attrs(int rhs_id, int alg, int dtype, const LaunchCfg& cfg,
                               cudaFuncAttributes* attr, int* blocks_per_sm);

// The mixed-batch kernel (batch_multi.cu): one persistent launch over items of three fixed
// kinds -- slot 0 Lorenz FP32 adaptive Tsit5, slot 1 Robertson FP32 Rosenbrock23,
// slot 2 GBM FP32 Euler-Maruyama, each without save times or step records -- its warps taking
// the items' queues in `order` (n entries, slot numbers), blocks of `block` (32..128) threads,
// as many as fit per SM.  mixed_slot gives an item's slot or -1.
int mixed_slot(int rhs_id, const ens_opts* o);
cudaError_t launch_mixed(const SolveArgs* const* by_slot, const int* order, int n, int block,
                         int num_sms, cudaStream_t s);

cudaError_t launch_philox(unsigned long long seed, long long index_offset, long long n_traj,
                          long long n_calls, unsigned int* out, cudaStream_t s);
cudaError_t launch_normals(unsigned long long seed, long long index_offset, long long n_traj,
                           long long n_per, int dtype, void* out, cudaStream_t s);

}  // namespace ens
