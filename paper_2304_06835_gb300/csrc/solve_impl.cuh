// solve_impl.cuh -- instantiation of the solve kernels for one (model, precision) pair and
// their launch configuration.  Included by the solve_<precision>_<model>.cu units.
#pragma once

#include <algorithm>

#include "ens_kernels.cuh"
#include "ens_pair.cuh"

namespace ens {

// Integrators with a paired (two trajectories per thread on FFMA2/FADD2/FMUL2) form.
template <class I>
struct PairOf {
  static constexpr bool ok = false;
};
template <class RHS>
struct PairOf<Adaptive<RHS, float, METH_TSIT5>> {
  static constexpr bool ok = RHS::autonomous && !RHS::has_event;
  typedef RHS rhs;
};

// Fixed-step integrators with a paired direct kernel (k_direct_pair).
template <class I>
struct DirectPairOf {
  static constexpr bool ok = false;
};
template <class RHS, int METH>
struct DirectPairOf<Fixed<RHS, float, METH>> {
  static constexpr bool ok =
      (METH == METH_FIX_TSIT5 || METH == METH_FIX_RK4) && RHS::autonomous && !RHS::has_event;
  typedef RHS rhs;
  static constexpr int meth = METH;
};

// dynamic shared memory of a launch (the dense saves' staging)
template <class I>
size_t dyn_smem(int block) {
  return (size_t)block * I::kSlotBytes;
}

template <class I, int TPT>
cudaError_t persistent_grid(const LaunchCfg& cfg, int* grid) {
  if (cfg.block > I::kMaxBlock) return cudaErrorLaunchOutOfResources;
  int bps = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_persistent<I, TPT>,
                                                                cfg.block, dyn_smem<I>(cfg.block));
  if (e != cudaSuccess) return e;
  if (bps == 0) return cudaErrorLaunchOutOfResources;  // the block does not fit an SM
  if (cfg.bps > 0) bps = std::min(bps, cfg.bps);
  else if (cfg.bps < 0) bps = std::max(1, (bps * -cfg.bps + 3) / 4);  // a quarter-step fraction
  *grid = std::max(1, bps) * cfg.num_sms;
  return cudaSuccess;
}

template <class RHS>
cudaError_t launch_persistent_pair(const SolveArgs& a, const LaunchCfg& cfg, cudaStream_t s) {
  int bps = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_persistent_pair<RHS>, cfg.block, 0);
  if (e != cudaSuccess) return e;
  if (bps == 0) return cudaErrorLaunchOutOfResources;  // the block does not fit an SM
  if (cfg.bps > 0) bps = std::min(bps, cfg.bps);
  else if (cfg.bps < 0) bps = std::max(1, (bps * -cfg.bps + 3) / 4);
  int grid = std::max(1, bps) * cfg.num_sms;
  const long long need = (a.N + 2LL * cfg.block - 1) / (2LL * cfg.block);
  grid = (int)std::min<long long>(grid, std::max<long long>(1, need));
  k_persistent_pair<RHS><<<grid, cfg.block, 0, s>>>(a);
  return cudaGetLastError();
}

template <class I, int TPT>
cudaError_t launch_persistent(const SolveArgs& a, const LaunchCfg& cfg, cudaStream_t s) {
  if constexpr (TPT == 2 && PairOf<I>::ok) {
    // two trajectories per thread in lockstep on the paired FP32 instructions (no save
    // times, no step record, no step cap)
    if (a.n_save == 0 && a.step_cap == 0 && !(a.dtmax_f < HUGE_VALF))
      return launch_persistent_pair<typename PairOf<I>::rhs>(a, cfg, s);
  }
  int grid = 0;
  cudaError_t e = persistent_grid<I, TPT>(cfg, &grid);
  if (e != cudaSuccess) return e;
  // never more resident threads than trajectory slots needed
  const long long need = (a.N + (long long)TPT * cfg.block - 1) / ((long long)TPT * cfg.block);
  grid = (int)std::min<long long>(grid, std::max<long long>(1, need));
  k_persistent<I, TPT><<<grid, cfg.block, dyn_smem<I>(cfg.block), s>>>(a);
  return cudaGetLastError();
}

template <class I>
cudaError_t launch_integ(const SolveArgs& a, const LaunchCfg& cfg, cudaStream_t s) {
  if (cfg.schedule == ENS_SCHED_DIRECT) {
    if constexpr (DirectPairOf<I>::ok) {
      // two trajectories per thread in lockstep on the paired FP32 instructions (final
      // state only)
      if (cfg.tpt == 2 && a.n_save == 0) {
        const long long pairs = (a.N + 2LL * cfg.block - 1) / (2LL * cfg.block);
        const int grid = (int)std::min<long long>(std::max<long long>(pairs, 1), 1LL << 30);
        typedef DirectPairOf<I> DP;
        k_direct_pair<typename DP::rhs, DP::meth><<<grid, cfg.block, 0, s>>>(a);
        return cudaGetLastError();
      }
    }
    const long long blocks = (a.N + cfg.block - 1) / cfg.block;
    const int grid = (int)std::min<long long>(blocks, 1LL << 30);
    if (cfg.block > I::kMaxBlock) return cudaErrorLaunchOutOfResources;
    k_direct<I><<<grid, cfg.block, dyn_smem<I>(cfg.block), s>>>(a);
    return cudaGetLastError();
  }
  if constexpr (I::kMaxTpt == 1) {  // one trajectory per thread whatever was asked
    return launch_persistent<I, 1>(a, cfg, s);
  } else {
    switch (cfg.tpt) {
      case 1: return launch_persistent<I, 1>(a, cfg, s);
      case 2: return launch_persistent<I, 2>(a, cfg, s);
      case 4: return launch_persistent<I, 4>(a, cfg, s);
    }
    return cudaErrorInvalidValue;
  }
}

template <class I>
cudaError_t attrs_integ(const LaunchCfg& cfg, cudaFuncAttributes* attr, int* bps) {
  const void* fn = nullptr;
  if (cfg.schedule == ENS_SCHED_DIRECT) {
    fn = (const void*)k_direct<I>;
    if constexpr (DirectPairOf<I>::ok)
      if (cfg.tpt == 2)
        fn = (const void*)k_direct_pair<typename DirectPairOf<I>::rhs, DirectPairOf<I>::meth>;
  } else if (cfg.tpt == 1 || I::kMaxTpt == 1) fn = (const void*)k_persistent<I, 1>;
  else if constexpr (I::kMaxTpt > 1) {
    if (cfg.tpt == 2) fn = (const void*)k_persistent<I, 2>;
    else if (cfg.tpt == 4) fn = (const void*)k_persistent<I, 4>;
    else return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaFuncGetAttributes(attr, fn);
  if (e != cudaSuccess) return e;
  if (cfg.block > I::kMaxBlock) {  // does not fit
    *bps = 0;
    return cudaSuccess;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fn, cfg.block,
                                                       dyn_smem<I>(cfg.block));
}

template <class I>
cudaError_t cost_keys_integ(const SolveArgs& a, CostScratch* cs, cudaStream_t s) {
  if (cs->keys)
    k_cost_values<I><<<cs->blocks, 256, 0, s>>>(a, cs->keys);
  else
    k_cost_keys<I><<<cs->blocks, 256, 0, s>>>(a, cs->bucket, cs->hist, cs->h0);
  return cudaGetLastError();
}

template <class I>
cudaError_t run_integ(const SolveArgs* a, const LaunchCfg& cfg, cudaStream_t s,
                      cudaFuncAttributes* attr, int* bps, CostScratch* cs) {
  if (cs) return cost_keys_integ<I>(*a, cs, s);
  return attr ? attrs_integ<I>(cfg, attr, bps) : launch_integ<I>(*a, cfg, s);
}

// Dispatch on the algorithm for one model: launch (attr == nullptr) or report attributes.
template <class RHS, class T>
cudaError_t dispatch_model(int alg, const SolveArgs* a, const LaunchCfg& cfg, cudaStream_t s,
                           bool* supported, cudaFuncAttributes* attr, int* bps,
                           CostScratch* cs) {
  *supported = true;
  if constexpr (RHS::stiff_only) {  // large stiff models: the Rosenbrock methods only
    if (alg == ENS_ROS23) return run_integ<Adaptive<RHS, T, METH_ROS23>>(a, cfg, s, attr, bps, cs);
    if (alg == ENS_RODAS4)
      return run_integ<Adaptive<RHS, T, METH_RODAS4>>(a, cfg, s, attr, bps, cs);
    if (alg == ENS_RODAS5P)
      return run_integ<Adaptive<RHS, T, METH_RODAS5P>>(a, cfg, s, attr, bps, cs);
  } else if constexpr (RHS::has_event) {  // events are located on the adaptive Tsit5 interpolant
    if (alg == ENS_TSIT5_ADAPTIVE) {
      if (a && a->step_cap > 0)
        return run_integ<Adaptive<RHS, T, METH_TSIT5_RECORD>>(a, cfg, s, attr, bps, cs);
      if (a && a->dense)
        return run_integ<Adaptive<RHS, T, METH_TSIT5_DENSE>>(a, cfg, s, attr, bps, cs);
      return run_integ<Adaptive<RHS, T, METH_TSIT5>>(a, cfg, s, attr, bps, cs);
    }
  } else if constexpr (RHS::sde_only) {
    if (alg == ENS_EM) return run_integ<Fixed<RHS, T, METH_FIX_EM>>(a, cfg, s, attr, bps, cs);
  } else {
    switch (alg) {
      case ENS_TSIT5_FIXED:
        return run_integ<Fixed<RHS, T, METH_FIX_TSIT5>>(a, cfg, s, attr, bps, cs);
      case ENS_TSIT5_ADAPTIVE:  // dense saving and the every-step record: variants of their own
        if (a && a->step_cap > 0)
          return run_integ<Adaptive<RHS, T, METH_TSIT5_RECORD>>(a, cfg, s, attr, bps, cs);
        if (a && a->dense)
          return run_integ<Adaptive<RHS, T, METH_TSIT5_DENSE>>(a, cfg, s, attr, bps, cs);
        return run_integ<Adaptive<RHS, T, METH_TSIT5>>(a, cfg, s, attr, bps, cs);
      case ENS_RK4: return run_integ<Fixed<RHS, T, METH_FIX_RK4>>(a, cfg, s, attr, bps, cs);
      case ENS_ROS23: return run_integ<Adaptive<RHS, T, METH_ROS23>>(a, cfg, s, attr, bps, cs);
      case ENS_RODAS4:
        return run_integ<Adaptive<RHS, T, METH_RODAS4>>(a, cfg, s, attr, bps, cs);
      case ENS_RODAS5P:
        return run_integ<Adaptive<RHS, T, METH_RODAS5P>>(a, cfg, s, attr, bps, cs);
      case ENS_EM:
        if constexpr (RHS::has_noise) {
          return run_integ<Fixed<RHS, T, METH_FIX_EM>>(a, cfg, s, attr, bps, cs);
        }
        break;
      case ENS_SIEA:
        if constexpr (DiagNoise<RHS>::value) {
          return run_integ<Fixed<RHS, T, METH_FIX_SIEA>>(a, cfg, s, attr, bps, cs);
        }
        break;
    }
  }
  *supported = false;
  return cudaSuccess;
}

}  // namespace ens

#define ENS_INSTANTIATE_MODEL(FN, MODEL, T)                                                 \
  namespace ens {                                                                           \
  cudaError_t FN(int alg, const SolveArgs* a, const LaunchCfg& cfg, cudaStream_t s,         \
                 bool* supported, cudaFuncAttributes* attr, int* bps, CostScratch* cs) {    \
    return dispatch_model<MODEL<T>, T>(alg, a, cfg, s, supported, attr, bps, cs);           \
  }                                                                                         \
  }
