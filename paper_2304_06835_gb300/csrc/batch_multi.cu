// batch_multi.cu -- the uneven batch in one persistent launch.
//
// The mixed batch of stiff, non-stiff and stochastic work (Sec. 6.4: divergent step counts
// under adaptive stepping) otherwise runs one persistent kernel per item, concurrently or one
// after another, and each kernel drains its own queue alone.  Here one resident grid serves
// all items: every warp runs the persistent loop of the first item in `order` until that
// item's queue is drained and its lanes are done, then moves on to the next item's queue, so
// while the first item's last trajectories finish on some warps, the others already work on
// the next item.  A warp only ever holds one item's kind of trajectory (no divergence between
// model codes), and the order is longest expected work first.  The kinds are fixed at compile
// time (the kernel holds the three integrators' code; its register budget is the largest of
// theirs).
#include <cstring>

#include "ens_internal.h"
#include "ens_kernels.cuh"
#include "ens_pair.cuh"

namespace ens {
namespace {

constexpr int kMixedSlots = 3;
typedef Adaptive<Robertson<float>, float, METH_ROS23> RobR23f;
typedef Fixed<GBM<float>, float, METH_FIX_EM> GbmEMf;

struct MixedArgs {
  SolveArgs a[kMixedSlots];  // by slot: Lorenz, Robertson, GBM
  int order[kMixedSlots];    // slots in processing order
  int n;
};

typedef Adaptive<Lorenz<float>, float, METH_TSIT5> LorTs5f;

// One trajectory per thread for every kind (the paired Lorenz loop took the union to 128
// registers); 110 registers, no spills.  Measured on the 10^6 mixed batch (3.44 ms with
// untuned item shapes against 4.28 ms for the serial kernels): register caps for 6 or 8 blocks
// of 128 per SM and out-of-line per-kind loops (each reading its arguments through a generic
// pointer) spill and were slower (3.62 - 4.51 ms).
__global__ void __launch_bounds__(128) k_persistent_mixed(const MixedArgs m) {
  for (int k = 0; k < m.n; ++k) {
    const int slot = m.order[k];  // uniform across the grid
    if (slot == 0)
      persistent_loop<LorTs5f, 1>(m.a[0]);
    else if (slot == 1)
      persistent_loop<RobR23f, 1>(m.a[1]);
    else
      persistent_loop<GbmEMf, 1>(m.a[2]);
  }
}

}  // namespace

int mixed_slot(int rhs_id, const ens_opts* o) {
  if (o->dtype != ENS_F32 || o->n_save != 0 || o->step_cap != 0) return -1;
  if (rhs_id == ENS_RHS_LORENZ && o->alg == ENS_TSIT5_ADAPTIVE && !(o->dtmax > 0)) return 0;
  if (rhs_id == ENS_RHS_ROBERTSON && o->alg == ENS_ROS23) return 1;
  if (rhs_id == ENS_RHS_GBM && o->alg == ENS_EM) return 2;
  return -1;
}

cudaError_t launch_mixed(const SolveArgs* const* by_slot, const int* order, int n, int block,
                         int num_sms, cudaStream_t s) {
  if (n < 1 || n > kMixedSlots || block < 32 || block > 128 || block % 32)
    return cudaErrorInvalidValue;
  MixedArgs m;
  std::memset(&m, 0, sizeof(m));
  for (int k = 0; k < n; ++k) {
    const int slot = order[k];
    if (slot < 0 || slot >= kMixedSlots || !by_slot[slot]) return cudaErrorInvalidValue;
    m.order[k] = slot;
    m.a[slot] = *by_slot[slot];
  }
  m.n = n;
  int bps = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_persistent_mixed, block, 0);
  if (e != cudaSuccess) return e;
  if (bps == 0) return cudaErrorLaunchOutOfResources;
  k_persistent_mixed<<<bps * num_sms, block, 0, s>>>(m);
  return cudaGetLastError();
}

}  // namespace ens
