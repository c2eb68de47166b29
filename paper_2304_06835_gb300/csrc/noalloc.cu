// noalloc.cu -- ens_solve_noalloc: the ensemble solve for callers that must not allocate.
//
// Some callers cannot let a library call cudaMalloc: code that runs while a framework owns
// every byte of device memory through its own pool, real-time loops where cudaMalloc's
// implicit device synchronisation is not acceptable, and plugins hosted by applications that
// forbid allocations after start-up.  This entry point keeps its scratch (the persistent
// queue counter, the cost-order permutation and bucket keys, the bucket cursors) in one
// file-scope device array of fixed size, so a call allocates nothing: the caller passes the
// inputs and outputs, as for ens_solve.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ens_internal.h"

namespace ens {
int set_last_error(int code, const char* msg);
}

using namespace ens;

namespace {

constexpr long long kMaxN = ENS_NOALLOC_MAX_N;
constexpr size_t kQueueOff = 0;                                  // 8 B counter
constexpr size_t kHistOff = 256;                                 // kCostBuckets x uint32
constexpr size_t kOrderOff = kHistOff + 4 * kCostBuckets;        // kMaxN x int32
constexpr size_t kBucketOff = kOrderOff + 4 * (size_t)kMaxN;     // kMaxN x uint16
constexpr size_t kScratchBytes = kBucketOff + 2 * (size_t)kMaxN;

// Every GPU that loads the library holds this array until the process exits.  All calls
// share it: each call clears the parts that must start at zero, and calls that overlap on
// the GPU (two streams, or two host threads) race on it.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_addr[kMaxDevices] = {};  // device address of g_scratch, per device

// Device address of g_scratch on the current device, looked up once per device.  In host
// code the name g_scratch is only a host-side stand-in and must never reach a kernel.
cudaError_t scratch_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = (unsigned char*)g_addr[dev];
  return cudaSuccess;
}

bool dims_of(int rhs_id, int* D, int* P) {
  switch (rhs_id) {
    case ENS_RHS_LORENZ: *D = 3; *P = 3; return true;
    case ENS_RHS_ROBERTSON: *D = 3; *P = 3; return true;
    case ENS_RHS_GBM: *D = 1; *P = 2; return true;
    case ENS_RHS_CRN: *D = 4; *P = 6; return true;
    case ENS_RHS_BALL: *D = 2; *P = 2; return true;
    case ENS_RHS_OREGO: *D = 3; *P = 3; return true;
    case ENS_RHS_HIRES: *D = 8; *P = 12; return true;
    case ENS_RHS_POLLU: *D = 20; *P = 25; return true;
  }
  return false;
}

bool fixed_alg(int alg) { return alg == ENS_TSIT5_FIXED || alg == ENS_RK4 || alg == ENS_EM; }

int check_args(int rhs_id, long long N, const void* params, const void* u0, const void* tspan,
               const ens_opts* o, const void* out) {
  int D, P;
  if (!dims_of(rhs_id, &D, &P)) return set_last_error(ENS_EINVAL, "unknown rhs_id");
  if (!o) return set_last_error(ENS_EINVAL, "null options");
  if (N < 0) return set_last_error(ENS_EINVAL, "N < 0");
  if (N > kMaxN)
    return set_last_error(ENS_EINVAL,
                          "ens_solve_noalloc: N exceeds ENS_NOALLOC_MAX_N (1048576 trajectories)");
  if (o->alg < ENS_TSIT5_FIXED || o->alg > ENS_EM) return set_last_error(ENS_EINVAL, "unknown algorithm");
  if (o->dtype != ENS_F32 && o->dtype != ENS_F64) return set_last_error(ENS_EINVAL, "unknown dtype");
  if (o->layout != ENS_LAYOUT_ROWMAJOR && o->layout != ENS_LAYOUT_SOA)
    return set_last_error(ENS_EINVAL, "unknown layout");
  if (o->alg == ENS_EM && rhs_id != ENS_RHS_GBM && rhs_id != ENS_RHS_CRN)
    return set_last_error(ENS_EINVAL, "Euler-Maruyama needs a model with noise (GBM, CRN)");
  if (rhs_id == ENS_RHS_CRN && o->alg != ENS_EM)
    return set_last_error(ENS_EINVAL, "the CRN model takes Euler-Maruyama only");
  if (rhs_id == ENS_RHS_BALL && o->alg != ENS_TSIT5_ADAPTIVE)
    return set_last_error(ENS_EINVAL, "the bouncing ball's events need adaptive Tsit5");
  if ((rhs_id == ENS_RHS_HIRES || rhs_id == ENS_RHS_POLLU) && o->alg != ENS_ROS23)
    return set_last_error(ENS_EINVAL, "HIRES and POLLU take Rosenbrock23 only");
  if (!std::isfinite(o->dtmax)) return set_last_error(ENS_EINVAL, "dtmax not finite");
  if (o->step_cap < 0) return set_last_error(ENS_EINVAL, "step_cap < 0");
  if (o->step_cap > 0 && (o->n_save > 0 || fixed_alg(o->alg)))
    return set_last_error(ENS_EINVAL, "step_cap needs an adaptive method and no save times");
  if (fixed_alg(o->alg) && !(o->dt > 0 && std::isfinite(o->dt)))
    return set_last_error(ENS_EINVAL, "fixed-step methods need a finite dt > 0");
  if (!fixed_alg(o->alg) && (!(o->abstol >= 1e-30) || !std::isfinite(o->abstol) ||
                             !(o->reltol >= 0) || !std::isfinite(o->reltol) ||
                             !std::isfinite(o->dt0)))
    return set_last_error(ENS_EINVAL, "tolerances or dt0 out of range");
  if (o->maxiters < 1 || o->maxiters > 2000000000LL)
    return set_last_error(ENS_EINVAL, "maxiters must be in [1, 2e9]");
  if (o->n_save < 0 || o->n_save > ENS_MAX_SAVE) return set_last_error(ENS_EINVAL, "n_save out of range");
  if (o->n_save > 0) {
    if (!o->saveat) return set_last_error(ENS_EINVAL, "saveat is NULL with n_save > 0");
    for (int i = 0; i < o->n_save; ++i)
      if (!std::isfinite(o->saveat[i]) || (i > 0 && o->saveat[i] < o->saveat[i - 1]))
        return set_last_error(ENS_EINVAL, "saveat must be finite and sorted");
  }
  if (o->schedule < ENS_SCHED_AUTO || o->schedule > ENS_SCHED_PERSISTENT)
    return set_last_error(ENS_EINVAL, "unknown schedule");
  if (o->block != 0 && (o->block < 32 || o->block > 1024 || o->block % 32 != 0))
    return set_last_error(ENS_EINVAL, "block must be 0 or a multiple of 32 in [32, 1024]");
  if (o->tpt != 0 && o->tpt != 1 && o->tpt != 2 && o->tpt != 4)
    return set_last_error(ENS_EINVAL, "tpt must be 0, 1, 2 or 4");
  if (o->refill_min < 0 || o->refill_min > 32) return set_last_error(ENS_EINVAL, "refill_min out of range");
  if (o->order < ENS_ORDER_AUTO || o->order > ENS_ORDER_COST) return set_last_error(ENS_EINVAL, "unknown order");
  if (N > 0 && (!params || !u0 || !tspan || !out)) return set_last_error(ENS_EINVAL, "null array");
  return ENS_OK;
}

}  // namespace

extern "C" int ens_solve_noalloc(int rhs_id, long long N, const void* params, const void* u0,
                                 const void* tspan, const ens_opts* o, void* out,
                                 signed char* status, int* stats, void* cuda_stream) {
  int rc = check_args(rhs_id, N, params, u0, tspan, o, out);
  if (rc) return rc;
  if (N == 0) return ENS_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && (dev < 0 || dev >= kMaxDevices)) e = cudaErrorInvalidDevice;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned char* base = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &base);
  if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));

  SolveArgs a;
  std::memset(&a, 0, sizeof(a));
  a.N = N;
  a.params = params;
  a.u0 = u0;
  a.tspan = tspan;
  a.out = out;
  a.status = status;
  a.stats = stats;
  a.layout = o->layout;
  a.n_save = o->n_save;
  a.dt = o->dt;
  a.abstol = o->abstol;
  a.reltol = o->reltol;
  a.dt0 = o->dt0;
  a.maxiters = o->maxiters;
  a.maxiters_i = (int)o->maxiters;
  a.abstol_f = (float)o->abstol;
  a.reltol_f = (float)o->reltol;
  a.dt0_f = (float)o->dt0;
  a.dtmax = o->dtmax > 0 ? o->dtmax : HUGE_VAL;
  a.step_cap = o->step_cap;
  a.step_t = o->step_t;
  a.step_n = o->step_n;
  a.dtmax_f = o->dtmax > 0 ? (float)o->dtmax : HUGE_VALF;
  a.refill_min = o->refill_min > 0 ? o->refill_min : 4;
  a.dense = o->dense != 0 && o->n_save > 0;
  a.seed = o->seed;
  a.index_offset = o->index_offset;
  a.queue = (unsigned long long*)(base + kQueueOff);
  a.order = nullptr;
  for (int i = 0; i < o->n_save; ++i) {
    a.saveat[i] = o->saveat[i];
    a.saveat_f[i] = (float)o->saveat[i];
  }

  LaunchCfg cfg;
  cfg.schedule = o->schedule != ENS_SCHED_AUTO
                     ? o->schedule
                     : (fixed_alg(o->alg) ? ENS_SCHED_DIRECT : ENS_SCHED_PERSISTENT);
  cfg.block = o->block ? o->block : 128;
  cfg.tpt = o->tpt ? o->tpt : 1;
  cfg.num_sms = sms;

  if (cfg.schedule == ENS_SCHED_PERSISTENT) {
    const bool cost =
        o->order == ENS_ORDER_COST || (o->order == ENS_ORDER_AUTO && !fixed_alg(o->alg));
    if (cost) {  // the bucket cursors are cleared inside launch_cost_order
      e = launch_cost_order(rhs_id, o->alg, o->dtype, a, (unsigned short*)(base + kBucketOff),
                            (unsigned int*)(base + kHistOff), (int*)(base + kOrderOff), s);
      if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));
      a.order = (const int*)(base + kOrderOff);
    }
    e = cudaMemsetAsync(base + kQueueOff, 0, sizeof(unsigned long long), s);  // queue from 0
    if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));
  }
  bool sup = false;
  e = launch_solve(rhs_id, o->alg, o->dtype, a, cfg, s, &sup);
  if (!sup) return set_last_error(ENS_ENOTSUP, "algorithm not available for this model");
  if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));
  return ENS_OK;
}
