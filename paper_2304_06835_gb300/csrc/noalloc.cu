// noalloc.cu -- ens_solve_noalloc: the ensemble solve for callers that must not allocate.
//
// Some callers cannot let a library call cudaMalloc: code that runs while a framework owns
// every byte of device memory through its own pool, real-time loops where cudaMalloc's
// implicit device synchronisation is not acceptable, and plugins hosted by applications that
// forbid allocations after start-up.  This entry point keeps its scratch (the persistent
// queue counter, the cost-order permutation and bucket keys, the bucket cursors) in one
// file-scope device array of fixed size, so a call allocates nothing: the caller passes the
// inputs and outputs, as for ens_solve.
#include <mutex>

#include "ens_internal.h"

using namespace ens;

namespace {

constexpr long long kMaxN = ENS_NOALLOC_MAX_N;
constexpr size_t kQueueOff = 0;                                  // 8 B counter
constexpr size_t kHistOff = 256;                                 // kCostHistWords x uint32
constexpr size_t kOrderOff = kHistOff + 4 * kCostHistWords;      // kMaxN x int32
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
// code the name g_scratch is only a host-side stand-in and must never reach a kernel.  The
// cached address belongs to the device's context: after cudaDeviceReset it is stale.
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

}  // namespace

extern "C" int ens_solve_noalloc(int rhs_id, long long N, const void* params, const void* u0,
                                 const void* tspan, const ens_opts* o, void* out,
                                 signed char* status, int* stats, void* cuda_stream) {
  // the checks of ens_solve, then the one limit of the fixed scratch
  int rc = validate_problem(rhs_id, N, params, u0, tspan, o, out);
  if (rc) return rc;
  if (N > kMaxN)
    return set_last_error(ENS_EINVAL,
                          "ens_solve_noalloc: N exceeds ENS_NOALLOC_MAX_N (1048576 trajectories)");
  if (N == 0) return ENS_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && (dev < 0 || dev >= kMaxDevices)) e = cudaErrorInvalidDevice;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned char* base = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &base);
  if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));

  // the same arguments, launch shape (explicit options, else the autotuner's cache, else the
  // defaults) and launch sequence as ens_solve; only the scratch is the fixed array
  SolveArgs a;
  fill_solve_args(&a, N, params, u0, tspan, o, out, status, stats);
  const LaunchCfg cfg = resolve_launch(rhs_id, N, o, sms);
  const SolveScratch sc{(unsigned long long*)(base + kQueueOff), (int*)(base + kOrderOff),
                        (unsigned short*)(base + kBucketOff), (unsigned int*)(base + kHistOff)};
  bool sup = false;
  // enqueue_solve clears the queue counter (and, for the longest-first order, the bucket
  // cursors) on the stream before the solve reads them
  e = enqueue_solve(rhs_id, o, a, cfg, sc, s, &sup);
  if (!sup) return set_last_error(ENS_ENOTSUP, "algorithm not available for this model");
  if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));
  return ENS_OK;
}
