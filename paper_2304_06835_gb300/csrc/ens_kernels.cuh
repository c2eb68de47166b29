// ens_kernels.cuh -- per-trajectory integrators and the fused ensemble kernels.
//
// One thread integrates one trajectory with the whole step loop in registers (the
// EnsembleGPUKernel design, Sec. 5.2 and its kernel listing: init, then step until t = tf,
// saving values).  Two schedules:
//   * direct:     thread i owns trajectories i, i + grid, ...
//   * persistent: a resident grid; whenever a lane finishes a trajectory it takes the next
//                 index from an atomic queue (warp-aggregated atomicAdd), so lanes of a warp
//                 whose trajectories need different step counts stay busy (the divergence
//                 of adaptive stepping noted in Sec. 6.4).  TPT slots per thread give ILP.
#pragma once

#include "ens_device.cuh"
#include "ens_internal.h"

namespace ens {

constexpr double kStopEps = 1e-12;    // remainder counted as having arrived (relative)
constexpr double kEta = 0.9;          // PI safety factor
constexpr float kLog2QoldInit = -13.287712379549449f;  // log2(1e-4)

// ------------------------------------------------------------------------------------------
// time accumulator: plain in FP64; Neumaier-compensated pair in FP32
template <class T>
struct Clock {
  T hi, lo;
  __device__ __forceinline__ void set(T v) { hi = v; lo = T(0); }
  __device__ __forceinline__ T value() const { return hi + lo; }
  __device__ __forceinline__ T remaining(T stop) const { return (stop - hi) - lo; }
  __device__ __forceinline__ void add(T h) {
    const T s = hi + h;
    const T c = (fabsf(hi) >= fabsf(h)) ? ((hi - s) + h) : ((h - s) + hi);
    lo += c;
    hi = s;
  }
  __device__ __forceinline__ void snap(bool cond, T v) {
    hi = cond ? v : hi;
    lo = cond ? T(0) : lo;
  }
};
template <>
struct Clock<double> {
  double hi;
  __device__ __forceinline__ void set(double v) { hi = v; }
  __device__ __forceinline__ double value() const { return hi; }
  __device__ __forceinline__ double remaining(double stop) const { return stop - hi; }
  __device__ __forceinline__ void add(double h) { hi += h; }
  __device__ __forceinline__ void snap(bool cond, double v) { hi = cond ? v : hi; }
};

// ------------------------------------------------------------------------------------------
// global-memory indexing for the two layouts
__device__ __forceinline__ long long in_idx(int layout, long long i, int k, long long N, int w) {
  return layout == ENS_LAYOUT_SOA ? (long long)k * N + i : i * w + k;
}
__device__ __forceinline__ long long out_idx(int layout, long long i, int s, int k, long long N,
                                             int S, int D) {
  return layout == ENS_LAYOUT_SOA ? ((long long)s * D + k) * N + i
                                  : (i * S + s) * (long long)D + k;
}

template <class T>
__device__ __forceinline__ T ldg(const void* base, long long idx) {
  return __ldg(static_cast<const T*>(base) + idx);
}

template <class T>
__device__ __forceinline__ T nan_of();
template <>
__device__ __forceinline__ float nan_of<float>() { return __int_as_float(0x7fc00000); }
template <>
__device__ __forceinline__ double nan_of<double>() {
  return __longlong_as_double(0x7ff8000000000000LL);
}

template <class RHS, class T>
__device__ __forceinline__ void load_problem(const SolveArgs& a, long long i, T* p, T* u, T& t0,
                                             T& tf) {
#pragma unroll
  for (int k = 0; k < RHS::P; ++k) p[k] = ldg<T>(a.params, in_idx(a.layout, i, k, a.N, RHS::P));
#pragma unroll
  for (int k = 0; k < RHS::D; ++k) u[k] = ldg<T>(a.u0, in_idx(a.layout, i, k, a.N, RHS::D));
  t0 = ldg<T>(a.tspan, in_idx(a.layout, i, 0, a.N, 2));
  tf = ldg<T>(a.tspan, in_idx(a.layout, i, 1, a.N, 2));
}

template <class RHS, class T>
__device__ __forceinline__ void write_slot(const SolveArgs& a, long long i, int s, const T* v) {
  const int S = a.n_save > 0 ? a.n_save : 1;
  T* o = static_cast<T*>(a.out);
#pragma unroll
  for (int k = 0; k < RHS::D; ++k) o[out_idx(a.layout, i, s, k, a.N, S, RHS::D)] = v[k];
}

__host__ __device__ constexpr int gcd_int(int a, int b) { return b == 0 ? a : gcd_int(b, a % b); }

template <class RHS, class T>
__device__ __forceinline__ void write_nan_slot(const SolveArgs& a, long long i, int s) {
  T v[RHS::D];
#pragma unroll
  for (int k = 0; k < RHS::D; ++k) v[k] = nan_of<T>();
  write_slot<RHS, T>(a, i, s, v);
}

__device__ __forceinline__ void write_stats(const SolveArgs& a, long long i, signed char st,
                                            int acc, int rej, int fev) {
  if (a.status) a.status[i] = st;
  if (a.stats) {
    a.stats[i] = acc;
    a.stats[a.N + i] = rej;
    a.stats[2 * a.N + i] = fev;
  }
}

// tolerances / first step in the solve's precision (FP32 solves read the FP32 copies)
template <class T>
struct Tol {
  static __device__ __forceinline__ T abstol(const SolveArgs& a) { return T(a.abstol); }
  static __device__ __forceinline__ T reltol(const SolveArgs& a) { return T(a.reltol); }
  static __device__ __forceinline__ T dt0(const SolveArgs& a) { return T(a.dt0); }
  static __device__ __forceinline__ T dtmax(const SolveArgs& a) { return T(a.dtmax); }
  static __device__ __forceinline__ T save(const SolveArgs& a, int s) { return T(a.saveat[s]); }
};
template <>
struct Tol<float> {
  static __device__ __forceinline__ float abstol(const SolveArgs& a) { return a.abstol_f; }
  static __device__ __forceinline__ float reltol(const SolveArgs& a) { return a.reltol_f; }
  static __device__ __forceinline__ float dt0(const SolveArgs& a) { return a.dt0_f; }
  static __device__ __forceinline__ float dtmax(const SolveArgs& a) { return a.dtmax_f; }
  static __device__ __forceinline__ float save(const SolveArgs& a, int s) { return a.saveat_f[s]; }
};

// Save times in shared memory, copied at block start by the kernels that run the adaptive
// integrators: lanes read them at their own save index, and a read of the kernel's parameter
// array at an index that differs across the warp is serialised over the distinct addresses.
// Dynamic shared memory of the kernels: the 16-byte staging of dense saves (Adaptive::put)
// and of the step record (Adaptive::record), one slot per thread.
extern __shared__ __align__(16) unsigned char ens_dyn_smem[];

template <class T>
__device__ __forceinline__ T* save_times_smem() {
  __shared__ T s[ENS_MAX_SAVE];
  return s;
}
template <class T>
__device__ __forceinline__ void load_save_times(const SolveArgs& a) {
  T* s = save_times_smem<T>();
  for (int k = threadIdx.x; k < a.n_save; k += blockDim.x) s[k] = Tol<T>::save(a, k);
  __syncthreads();
}

template <class T>
__device__ __forceinline__ T rms_scaled(const T* x, const T* sc, int D) {
  T s = T(0);
  for (int j = 0; j < D; ++j) {
    const T r = x[j] / sc[j];
    s = M<T>::fma(r, r, s);
  }
  return M<T>::sqrt(s / T(D));
}

// ------------------------------------------------------------------------------------------
// Adaptive integrators: Tsit5 with PI control (Sec. 3.1) and Rosenbrock23 (Sec. 3.2.1).
// METH_TSIT5_DENSE is Tsit5 whose save times take the dense output of the step that covers
// them instead of cutting the steps (the steps are those of the solve without save times);
// METH_TSIT5_RECORD is Tsit5 that records every accepted step.  Each variant carries only
// its own output code: the record's staging in the dense kernel cost it 12 registers and
// ~10 %.
enum {
  METH_TSIT5 = 0, METH_ROS23 = 1, METH_TSIT5_DENSE = 2, METH_TSIT5_RECORD = 3, METH_RODAS4 = 4,
  METH_RODAS5P = 5
};

template <class RHS, class T, int METH>
struct Adaptive {
  static constexpr int D = RHS::D, P = RHS::P;
  static constexpr bool kDense = METH == METH_TSIT5_DENSE;
  static constexpr bool kRecord = METH == METH_TSIT5_RECORD;
  // the every-step record: staged (kRecord) or with scalar stores (Rosenbrock23); the plain
  // Tsit5 variant never records (Tsit5 records run on METH_TSIT5_RECORD)
  // Rosenbrock methods: Rosenbrock23, Rodas4, Rodas5P (no dense output, no events)
  static constexpr bool kRos = METH == METH_ROS23 || METH == METH_RODAS4 || METH == METH_RODAS5P;
  static constexpr bool kRodas = METH == METH_RODAS4 || METH == METH_RODAS5P;
  static constexpr bool kHasRecord = kRecord || kRos;
  static constexpr bool kEvent = RHS::has_event && !kRos;
  static constexpr bool kKeepStages = kDense || kEvent;  // stages 2..6 outlive the step
  // trajectories per thread (dense saving and the record: one, the staging slot is the
  // thread's)
  static constexpr int kMaxTpt =
      (RHS::stiff_only || kRodas || METH == METH_TSIT5_DENSE || METH == METH_TSIT5_RECORD) ? 1
                                                                                          : 4;
  // Dense saving stages kSaveK saves (a whole number of 16-byte words) per lane in shared
  // memory and writes them with vector stores when the output is trajectory-major, 16-byte
  // aligned and n_save is a multiple of kSaveK: the lanes of a warp save at different times,
  // so scalar stores would reach L2 as 4- or 8-byte pieces of separate sectors.  (Staged in
  // registers the group stayed live through the whole solve: 12 registers and ~8 %.)
  static constexpr int kRowBytes = D * int(sizeof(T));
  static constexpr int kRowK = 16 / gcd_int(16, kRowBytes);  // rows in whole 16-byte words
  static constexpr int kSaveK = kDense ? kRowK : 1;
  static constexpr int kSaveWords = kSaveK * kRowBytes / 16;
  // The every-step record (kRecord) stages kRecK entries in shared memory likewise: whole
  // 16-byte words of states and of times.
  static constexpr int kTimeK = 16 / int(sizeof(T));
  static constexpr int kRecK =
      kRecord ? kRowK * kTimeK / gcd_int(kRowK, kTimeK) : 1;  // lcm of the two groups
  // staged values per thread (the thread's slot: whole 16-byte words of saves, or of record
  // states then times; a runtime stride between slots kept a dozen addresses live), and the
  // largest block, which keeps the staging and the save times under the default 48 KB
  static constexpr int kStageElems = kDense ? kSaveK * D : kRecord ? kRecK * (D + 1) : 0;
  static constexpr int kMaxBlock = (kDense || kRecord) ? 512 : 1024;
  // Slot stride: an odd number of 16-byte words, so the 16-byte reads of 8 consecutive lanes
  // cover all 32 banks once (an even count, e.g. the record's 64 bytes, put every lane's
  // 4-byte stores into two banks: 16-way conflicts).
  static constexpr int kSlotBytes0 = kStageElems * int(sizeof(T));
  static constexpr int kSlotBytes =
      (kSlotBytes0 > 0 && (kSlotBytes0 / 16) % 2 == 0) ? kSlotBytes0 + 16 : kSlotBytes0;
  // controller exponents: beta1 = 0.7/k, beta2 = 0.4/k, reject exponent 1/k, with k the error
  // estimate's order + 1 (Tsit5 5(4) and Rodas5P 5(4): 5, Rodas4 4(3): 4, Rosenbrock23: 3);
  // the starting step takes the advancing solution's order
  static constexpr float kOrd =
      METH == METH_ROS23 ? 3.f : METH == METH_RODAS4 ? 4.f : 5.f;
  static constexpr int kInitOrder = METH == METH_ROS23 ? 2 : METH == METH_RODAS4 ? 4 : 5;
  // f evaluations per attempt: Tsit5 6 (FSAL), Rosenbrock23 2 (FSAL), Rodas: stages 2..S and
  // f(u_{n+1})
  static constexpr int kStepsPerAdvance = 1;  // attempts one advance() can make
  static constexpr int kFevPerAttempt = METH == METH_ROS23 ? 2
                                        : METH == METH_RODAS4 ? Rodas4Tab::S
                                        : METH == METH_RODAS5P ? Rodas5PTab::S : 6;
  using Real = T;
  static constexpr bool kSmemSaves = true;  // reads save times from save_times_smem

  T u[D], fk[D], p[P];
  Clock<T> t;
  T tf, h;
  T stop, stop_thr;   // next stop (a save time before tf, or tf) and its arrival threshold
  float lq;           // log2 q_{n-1}
  int attempts, rejected, si, fev0, nev;  // nev: events handled (one extra f each)
  int st;             // ENS_TRAJ_* (int, not char: no byte packing in the loop)
  int stop_is_save;
  T nsv;  // dense: the next save time (+inf past the last)
  long long idx;
  bool stage;                       // this solve stages its saves (see kSaveK)
  bool rstage;                      // this solve stages its record (see kRecK)

  // write save slot si (then ++si): directly, or through the 16-byte staging
  __device__ __forceinline__ void put(const SolveArgs& a, const T* v) {
    if constexpr (kDense) {
      if (stage) {
        const int k = si % kSaveK;
        T* sl = reinterpret_cast<T*>(ens_dyn_smem + threadIdx.x * kSlotBytes);
#pragma unroll
        for (int j = 0; j < D; ++j) sl[k * D + j] = v[j];
        if (k == kSaveK - 1) {  // a full group: slots si - k .. si
          uint4* o = reinterpret_cast<uint4*>(static_cast<T*>(a.out) +
                                              (idx * a.n_save + (si - k)) * (long long)D);
          const uint4* w = reinterpret_cast<const uint4*>(sl);
#pragma unroll
          for (int q = 0; q < kSaveWords; ++q) o[q] = w[q];
        }
        ++si;
        return;
      }
    }
    write_slot<RHS, T>(a, idx, si, v);
    ++si;
  }
  __device__ __forceinline__ void put_nan(const SolveArgs& a) {
    T v[D];
#pragma unroll
    for (int j = 0; j < D; ++j) v[j] = nan_of<T>();
    put(a, v);
  }

  __device__ __forceinline__ void set_stop(const SolveArgs& a) {
    stop_is_save = !kDense && si < a.n_save && save_times_smem<T>()[si] < tf;
    stop = stop_is_save ? save_times_smem<T>()[si] : tf;
    stop_thr = T(kStopEps) * M<T>::max(T(1), M<T>::abs(stop));
  }

  // kRec = false compiles the every-step record and the save times out (for the paired
  // kernel, which the host launches with neither: dead code there still cost it a register
  // and ~3 %)
  template <bool kRec = true>
  __device__ __forceinline__ void init(long long i, const SolveArgs& a) {
    idx = i;
    T t0;
    load_problem<RHS, T>(a, i, p, u, t0, tf);
    t.set(t0);
    RHS::f(u, p, t0, fk);
    fev0 = 1;
    if (Tol<T>::dt0(a) > T(0)) {
      h = Tol<T>::dt0(a);
    } else {  // the ordering pre-pass may have formed it already (the same arithmetic)
      h = a.h0 ? ldg<T>(a.h0, i) : initial_step(a, t0);
      fev0 = 2;
    }
    lq = kLog2QoldInit;
    attempts = 0;
    rejected = 0;
    nev = 0;
    st = ENS_TRAJ_OK;
    si = 0;
    stage = kDense && a.layout == ENS_LAYOUT_ROWMAJOR && a.n_save % kSaveK == 0 &&
            (reinterpret_cast<unsigned long long>(a.out) & 15ull) == 0;
    rstage = kRecord && a.step_cap > 0 && a.layout == ENS_LAYOUT_ROWMAJOR &&
             a.step_cap % kRecK == 0 && a.step_t != nullptr &&
             ((reinterpret_cast<unsigned long long>(a.out) |
               reinterpret_cast<unsigned long long>(a.step_t)) & 15ull) == 0;
    if constexpr (kRec) {
      while (si < a.n_save && save_times_smem<T>()[si] < t0) put_nan(a);
      if (kDense)  // save times at t0 take u0; the steps then run to tf uncut
        while (si < a.n_save && save_times_smem<T>()[si] == t0 && t0 <= tf) put(a, u);
      if (kDense) next_save(a);
      if (kHasRecord && a.step_cap > 0) record(a, 0, t0);
      set_stop(a);
    } else {  // no save times: the only stop is tf
      stop_is_save = 0;
      stop = tf;
      stop_thr = T(kStopEps) * M<T>::max(T(1), M<T>::abs(tf));
    }
  }

  // every-step record: entry k = (t, u) after k accepted steps, k < step_cap
  __device__ __forceinline__ void record(const SolveArgs& a, int k, T tk) {
    if (k >= a.step_cap) return;
    if constexpr (kRecord) {
      if (rstage) {  // stage; a full group of kRecK entries goes out as 16-byte stores
        const int q = k % kRecK;
        T* sbuf = reinterpret_cast<T*>(ens_dyn_smem + threadIdx.x * kSlotBytes);  // states
        T* tbuf = sbuf + kRecK * D;                                                // times
#pragma unroll
        for (int j = 0; j < D; ++j) sbuf[q * D + j] = u[j];
        tbuf[q] = tk;
        if (q == kRecK - 1) {
          uint4* ou = reinterpret_cast<uint4*>(static_cast<T*>(a.out) +
                                               (idx * a.step_cap + (k - q)) * (long long)D);
          uint4* ot = reinterpret_cast<uint4*>(static_cast<T*>(a.step_t) + idx * a.step_cap +
                                               (k - q));
          const uint4* wu = reinterpret_cast<const uint4*>(sbuf);
          const uint4* wt = reinterpret_cast<const uint4*>(tbuf);
#pragma unroll
          for (int w = 0; w < kRecK * kRowBytes / 16; ++w) ou[w] = wu[w];
#pragma unroll
          for (int w = 0; w < kRecK * int(sizeof(T)) / 16; ++w) ot[w] = wt[w];
        }
        return;
      }
    }
    T* o = static_cast<T*>(a.out);
#pragma unroll
    for (int j = 0; j < D; ++j) o[out_idx(a.layout, idx, k, j, a.N, a.step_cap, D)] = u[j];
    if (a.step_t)
      static_cast<T*>(a.step_t)[a.layout == ENS_LAYOUT_SOA ? (long long)k * a.N + idx
                                                             : idx * a.step_cap + k] = tk;
  }

  // dense output: every save time in (t_n, t_n + lim] of the accepted step (lim = hs, or the
  // event's offset when an event ends the step early), theta = (s - t_n) / hs on the
  // compensated clock; a save at the end of the last step is u_{n+1}.  The interpolant is
  // evaluated from its coefficients in theta (dense_coeffs, formed once per step and only by
  // a lane with a save in it): 4 FMA per component and save instead of the 7 weights.
  __device__ __forceinline__ bool dense_pending(const SolveArgs& a, T lim, bool last) const {
    return nsv <= tf && ((last && nsv == stop) || t.remaining(nsv) <= lim);
  }
  __device__ __forceinline__ void next_save(const SolveArgs& a) {
    nsv = si < a.n_save ? save_times_smem<T>()[si] : T(INFINITY);
  }
  __device__ __forceinline__ void dense_saves(const SolveArgs& a, const T (*cq)[D], T hs, T lim,
                                              bool last, const T* unew) {
    while (si < a.n_save) {
      const T sv = save_times_smem<T>()[si];
      if (sv > tf) break;
      const T rs = t.remaining(sv);
      const bool at_end = last && sv == stop;
      if (!at_end && rs > lim) break;
      if (at_end) {
        put(a, unew);
      } else {
        T w[D];
        dense_poly<RHS, T>(u, cq, M<T>::fast_div(rs, hs), w);
        put(a, w);
      }
    }
    next_save(a);
  }

  // Hairer-Norsett-Wanner I, II.4: starting step size (a heuristic: the FP32 solve forms it
  // with fast division and MUFU-based pow)
  __device__ __forceinline__ T initial_step(const SolveArgs& a, T t0) {
    T sc[D], u1[D], f1[D];
    const T atol = Tol<T>::abstol(a), rtol = Tol<T>::reltol(a);
    T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      sc[j] = M<T>::fast_div(T(1), M<T>::fma(rtol, M<T>::abs(u[j]), atol));
      s0 = M<T>::fma(u[j] * sc[j], u[j] * sc[j], s0);
      s1 = M<T>::fma(fk[j] * sc[j], fk[j] * sc[j], s1);
    }
    const T d0 = M<T>::sqrt(s0 * T(1.0 / D)), d1 = M<T>::sqrt(s1 * T(1.0 / D));
    const T h0 = (d0 < T(1e-5) || d1 < T(1e-5)) ? T(1e-6) : T(0.01) * M<T>::fast_div(d0, d1);
#pragma unroll
    for (int j = 0; j < D; ++j) u1[j] = M<T>::fma(h0, fk[j], u[j]);
    RHS::f(u1, p, t0 + h0, f1);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const T v = (f1[j] - fk[j]) * sc[j];
      s2 = M<T>::fma(v, v, s2);
    }
    const T d2 = M<T>::fast_div(M<T>::sqrt(s2 * T(1.0 / D)), h0);
    const T dm = M<T>::max(d1, d2);
    const T h1 = (dm <= T(1e-15)) ? M<T>::max(T(1e-6), h0 * T(1e-3))
                                  : M<T>::fast_pow(M<T>::fast_div(T(0.01), dm),
                                                   T(1.0 / (kInitOrder + 1)));
    return M<T>::min(T(100) * h0, h1);
  }

  // one attempt; returns true when the trajectory is finished.  The common path has no
  // data-dependent branch: the rare exits are merged into one test and accept/reject is
  // applied with selects.
  __device__ __forceinline__ bool advance(const SolveArgs& a) {
    T rem = t.remaining(stop);
    if (rem <= stop_thr) {  // arrived at the stop
      do {
        t.set(stop);
        if (!stop_is_save) {  // tf (dense: every save left within the arrival threshold)
          while (si < a.n_save &&
                 (save_times_smem<T>()[si] == tf || (kDense && save_times_smem<T>()[si] <= tf)))
            put(a, u);
          return true;
        }
        put(a, u);
        set_stop(a);
        rem = t.remaining(stop);
      } while (rem <= stop_thr);
    }
    // the cap (+inf when not set) keeps a NaN step NaN, so a failing trajectory fails alike
    // with and without it
    const T dtmax = Tol<T>::dtmax(a);
    const T hcap = (h > dtmax) ? dtmax : h;
    const bool last = hcap >= rem;
    const T hs = last ? rem : hcap;
    const T tnow = t.value();
    const bool capped = attempts >= a.maxiters_i;
    const bool tiny = hs < T(M<T>::dtmin_factor) * M<T>::max(T(1), M<T>::abs(tnow));
    T unew[D], es[D], fnew[D], kmid[kKeepStages ? 5 * D : 1];
    if constexpr (METH == METH_ROS23)
      ros23_step<RHS, T>(u, p, tnow, hs, fk, unew, es, fnew);
    else if constexpr (METH == METH_RODAS4)
      rodas_step<RHS, T, Rodas4Tab>(u, p, tnow, hs, fk, unew, es, fnew);
    else if constexpr (METH == METH_RODAS5P)
      rodas_step<RHS, T, Rodas5PTab>(u, p, tnow, hs, fk, unew, es, fnew);
    else
      tsit5_step<RHS, T, true>(u, p, tnow, hs, fk, unew, es, fnew, kKeepStages ? kmid : nullptr);
    // q^2 = (1/D) sum_j (E_j / (atol + rtol max(|u_j|, |unew_j|)))^2 with E_j = h es_j
    // (the Rodas steps return E_j itself).
    // The ratios are formed in FP32 for both precisions (E itself is accumulated in T).
    const T atol = Tol<T>::abstol(a), rtol = Tol<T>::reltol(a);
    float r2 = 0.f;
    bool fin = true;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const T sc = M<T>::fma(rtol, M<T>::max(M<T>::abs(u[j]), M<T>::abs(unew[j])), atol);
      const float r = __fdividef(float(kRodas ? es[j] : hs * es[j]), float(sc));  // Rodas: E itself
      r2 = __fmaf_rn(r, r, r2);
      fin = fin && M<T>::finite(unew[j]);
    }
    const float q2 = r2 * (1.f / float(D));
    if (capped || tiny || !fin || isnan(q2)) {
      // priority as the checks would run in sequence: cap, step too small, non-finite attempt
      st = capped ? ENS_TRAJ_MAXITERS : (tiny ? ENS_TRAJ_DT_MIN : ENS_TRAJ_NONFINITE);
      attempts += (capped || tiny) ? 0 : 1;
      return true;
    }
    ++attempts;
    const bool acc = q2 <= 1.f;
    T th_ev = T(-1);
    if constexpr (kEvent) {
      if (acc) {
        T cq[4][D];
        dense_coeffs<RHS, T>(hs, fk, kmid, fnew, cq);
        th_ev = find_event<RHS, T>(u, unew, p, tnow, hs, cq);
        if (th_ev > T(0)) {  // the event: saves up to it from this step, state, affect, f
          const bool cut = th_ev < T(1);
          if (kDense) dense_saves(a, cq, hs, cut ? th_ev * hs : hs, last && !cut, unew);
          if (cut) dense_poly<RHS, T>(u, cq, th_ev, unew);
          RHS::event_affect(unew, p, tnow + th_ev * hs);
          RHS::f(unew, p, tnow + th_ev * hs, fnew);
          ++nev;
        }
      }
    }
    if constexpr (kDense) {
      if (acc && !(th_ev > T(0)) && dense_pending(a, hs, last)) {
        T cq[4][D];
        dense_coeffs<RHS, T>(hs, fk, kmid, fnew, cq);
        dense_saves(a, cq, hs, hs, last, unew);
      }
    }
    const bool cut = th_ev > T(0) && th_ev < T(1);  // an event ended the step early
    // PI control: accept fac = eta q_n^{-beta1} q_{n-1}^{beta2} in [0.2, 10];
    // reject fac = max(0.2, eta q_n^{-1/k}).  Exponentials in log2 form (q guarded at 1e-10).
    const float L = lg2_approx(fmaxf(q2, 1e-20f));  // log2 q^2
    const float e = acc ? __fmaf_rn(-0.35f / kOrd, L, (0.4f / kOrd) * lq) : (-0.5f / kOrd) * L;
    const float fac = fminf(acc ? 10.f : 1.f, fmaxf(0.2f, float(kEta) * ex2_approx(e)));
#pragma unroll
    for (int j = 0; j < D; ++j) {
      u[j] = acc ? unew[j] : u[j];
      fk[j] = acc ? fnew[j] : fk[j];
    }
    t.add(acc ? (cut ? th_ev * hs : hs) : T(0));
    t.snap(acc && last && !cut, stop);
    lq = acc ? fmaxf(0.5f * L, kLog2QoldInit) : lq;
    rejected += acc ? 0 : 1;
    if constexpr (kHasRecord)
      if (a.step_cap > 0 && acc) record(a, attempts - rejected, t.value());
    h = hs * T(fac);
    return false;
  }

  template <bool kRec = true>
  __device__ __forceinline__ void finish(const SolveArgs& a) {
    if (!kRec) {
      write_slot<RHS, T>(a, idx, 0, u);
    } else {
      if (a.n_save == 0 && a.step_cap == 0) write_slot<RHS, T>(a, idx, 0, u);
      while (si < a.n_save) put_nan(a);
    }
    if constexpr (kRecord && kRec) {
      if (rstage) {  // the staged entries of an unfinished last group, with scalar stores
        const int n = attempts - rejected + 1 < a.step_cap ? attempts - rejected + 1
                                                           : a.step_cap;
        const int k0 = n - n % kRecK;
        T* o = static_cast<T*>(a.out);
        T* ot = static_cast<T*>(a.step_t);
        const T* sbuf = reinterpret_cast<const T*>(ens_dyn_smem + threadIdx.x * kSlotBytes);
        const T* tbuf = sbuf + kRecK * D;
#pragma unroll
        for (int g = 0; g < kRecK; ++g)
          if (k0 + g < n) {
#pragma unroll
            for (int j = 0; j < D; ++j) o[(idx * a.step_cap + k0 + g) * D + j] = sbuf[g * D + j];
            ot[idx * a.step_cap + k0 + g] = tbuf[g];
          }
      }
    }
    if (kRec && a.step_n) a.step_n[idx] = attempts - rejected + 1;
    write_stats(a, idx, st, attempts - rejected, rejected,
                fev0 + kFevPerAttempt * attempts + nev);
  }

  // expected work of trajectory i: (tf - t0) / (starting step), the number of steps a solve
  // that kept the Hairer-Norsett-Wanner starting step would take
  // (h0c: when not null, the starting step is kept there for the solve's initialisation)
  static __device__ __forceinline__ float cost_key(const SolveArgs& a, long long i, void* h0c) {
    Adaptive s;
    T t0;
    load_problem<RHS, T>(a, i, s.p, s.u, t0, s.tf);
    RHS::f(s.u, s.p, t0, s.fk);
    const T h0 = s.initial_step(a, t0);
    if (h0c) static_cast<T*>(h0c)[i] = h0;
    return float(s.tf - t0) / float(h0);
  }
};

// ------------------------------------------------------------------------------------------
// Fixed-step integrators: Tsit5, RK4 and Euler-Maruyama.
// n = ceil((tf - t0)/dt - 1e-12) steps; h = dt except the last, h = tf - (t0 + (n-1) dt).
enum { METH_FIX_TSIT5 = 0, METH_FIX_RK4 = 1, METH_FIX_EM = 2, METH_FIX_SIEA = 3 };

// models whose noise is diagonal (component j driven by W_j through b_j(u)) expose diag_b
template <class R, class = void>
struct DiagNoise : std::false_type {};
template <class R>
struct DiagNoise<R, std::void_t<decltype(&R::diag_b)>> : std::true_type {};

constexpr long long kMaxFixedSteps = 0x7ffffffeLL;  // steps of one fixed-step trajectory

template <class RHS, class T, int METH>
struct Fixed {
  using Real = T;
  static constexpr bool kSmemSaves = false;
  static constexpr int kStageElems = 0, kSlotBytes = 0, kMaxBlock = 1024;
  static constexpr int D = RHS::D, P = RHS::P;
  // Euler-Maruyama step k uses normals k*NW .. k*NW + NW - 1 of the trajectory's stream: one
  // Philox call serves kSub steps (NW <= per_call) or one step takes kCalls calls.
  static constexpr int kNW = RHS::NW > 0 ? RHS::NW : 1, kPC = Normals<T>::per_call;
  static_assert(kPC % kNW == 0 || kNW % kPC == 0, "normals per step vs per Philox call");
  static constexpr int kMaxTpt = 4;
  static constexpr bool kSde = METH == METH_FIX_EM || METH == METH_FIX_SIEA;
  static constexpr int kSub = (kSde && kNW <= kPC) ? kPC / kNW : 1;
  static constexpr int kCalls = (kSde && kNW > kPC) ? kNW / kPC : 1;
  static constexpr int kStepsPerAdvance = kSde ? kSub : 1;  // one Philox call serves kSub steps

  T u[D], fk[D], p[P];
  T h_reg, h_last, t0f;
  // SDE steps: sqrt(h) and 1/(4 sqrt(h)) of the regular and of the last step, formed once per
  // trajectory (the same values the steps would form)
  T sq_reg, sq_last, q4_reg, q4_last;
  double t0, tf;
  int n, nrun, k, next_ks;  // step counts in 32 bits (the 64-bit ones cost ~7 % on GBM EM)
  int si;
  long long idx;

  __device__ __forceinline__ int ks_of(const SolveArgs& a, int s) const {
    const double sv = a.saveat[s];
    if (sv < t0 || sv > tf) return -1;
    long long ks = (sv <= t0) ? 0 : (long long)ceil((sv - t0) / a.dt - 1e-12);
    return ks < 0 ? 0 : (ks > n ? n : ks);
  }

  __device__ __forceinline__ void advance_saves(const SolveArgs& a) {
    // record every save whose step index has been reached; NaN for out-of-range ones
    while (si < a.n_save) {
      if (next_ks < 0) {
        write_nan_slot<RHS, T>(a, idx, si);
      } else if (next_ks == k) {
        write_slot<RHS, T>(a, idx, si, u);
      } else {
        break;
      }
      ++si;
      if (si < a.n_save) next_ks = ks_of(a, si);
    }
  }

  __device__ __forceinline__ void init(long long i, const SolveArgs& a) {
    idx = i;
    T t0t, tft;
    load_problem<RHS, T>(a, i, p, u, t0t, tft);
    t0f = t0t;
    t0 = double(t0t);
    tf = double(tft);
    long long n64 = (tf > t0) ? (long long)ceil((tf - t0) / a.dt - 1e-12) : 0;
    if (n64 < 0) n64 = 0;
    // at most kMaxFixedSteps steps per trajectory: a longer span stops there, MAXITERS
    long long r64 = n64 < a.maxiters ? n64 : a.maxiters;
    r64 = r64 < kMaxFixedSteps ? r64 : kMaxFixedSteps;
    n = int(n64 <= kMaxFixedSteps ? n64 : kMaxFixedSteps + 1);
    nrun = int(r64);
    h_reg = T(a.dt);
    h_last = n64 > 0 ? T(tf - (t0 + double(n64 - 1) * a.dt)) : T(0);
    if constexpr (kSde) {
      sq_reg = M<T>::sqrt(h_reg);
      sq_last = M<T>::sqrt(h_last);
      q4_reg = T(0.25) / sq_reg;
      q4_last = T(0.25) / sq_last;
    }
    k = 0;
    if (METH == METH_FIX_TSIT5) RHS::f(u, p, t0t, fk);
    si = 0;
    if (a.n_save > 0) {
      next_ks = ks_of(a, 0);
      advance_saves(a);
    }
  }

  // kReg: the caller knows this is not the trajectory's last step (h = h_reg)
  template <bool kReg = false>
  __device__ __forceinline__ void one_step(const SolveArgs& a, const T* z) {
    const bool lastk = !kReg && k == n - 1;
    const T h = lastk ? h_last : h_reg;
    const T tk = T(kSde || !RHS::autonomous ? t0f + T(k) * h_reg : T(0));
    T unew[D];
    if (METH == METH_FIX_TSIT5) {
      T k7[D];
      tsit5_step<RHS, T, false>(u, p, tk, h, fk, unew, nullptr, k7);
#pragma unroll
      for (int j = 0; j < D; ++j) fk[j] = k7[j];
    } else if (METH == METH_FIX_RK4) {
      rk4_step<RHS, T>(u, p, tk, h, unew);
    } else if (METH == METH_FIX_SIEA) {
      siea_step(u, p, tk, h, lastk ? sq_last : sq_reg, lastk ? q4_last : q4_reg, z, unew);
    } else {
      em_step(u, p, tk, h, lastk ? sq_last : sq_reg, z, unew);
    }
#pragma unroll
    for (int j = 0; j < D; ++j) u[j] = unew[j];
    ++k;
    if (a.n_save > 0) advance_saves(a);
  }

  template <class R = RHS>
  __device__ __forceinline__ typename std::enable_if<R::has_noise>::type em_step(
      const T* uu, const T* pp, T tk, T h, T sq, const T* z, T* unew) {  // sq = sqrt(h)
    T dr[D], nz[D];
    RHS::sde(uu, pp, tk, sq, z, dr, nz);
    // increment first (a h + sum_m b_m sqrt(h) Z_m), then one rounding at the scale of X
#pragma unroll
    for (int j = 0; j < D; ++j) unew[j] = uu[j] + M<T>::fma(dr[j], h, nz[j]);
  }
  template <class R = RHS>
  __device__ __forceinline__ typename std::enable_if<!R::has_noise>::type em_step(
      const T*, const T*, T, T, T, const T*, T*) {}

  // Weak order 2 stochastic Runge-Kutta step (GPUSIEA, Sec. 5.2.2; the improved-Euler-type
  // member of the SRK family of Sec. 3.3), diagonal noise, dW_j = sqrt(h) Z_j:
  //   Ybar = X + a h + b dW,  Y+- = X + a h +- b sqrt(h),
  //   X1 = X + (a(X) + a(Ybar)) h/2 + (b(Y+) + b(Y-) + 2 b(X)) dW/4
  //        + (b(Y+) - b(Y-)) (dW^2 - h) / (4 sqrt(h)).
  // (sq = sqrt(h) and q4 = 0.25 / sq, formed once per trajectory)
  template <class R = RHS>
  __device__ __forceinline__ typename std::enable_if<DiagNoise<R>::value>::type siea_step(
      const T* uu, const T* pp, T tk, T h, T sq, T q4, const T* z, T* unew) {
    typedef M<T> m;
    T a0[D], a1[D], b0[D], bp[D], bm[D], Y[D], dW[D], ah[D];
    RHS::f(uu, pp, tk, a0);
    RHS::diag_b(uu, pp, tk, b0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      dW[j] = sq * z[j];
      ah[j] = m::fma(a0[j], h, uu[j]);  // X + a h
      Y[j] = m::fma(b0[j], dW[j], ah[j]);
    }
    RHS::f(Y, pp, tk + h, a1);
#pragma unroll
    for (int j = 0; j < D; ++j) Y[j] = m::fma(b0[j], sq, ah[j]);
    RHS::diag_b(Y, pp, tk + h, bp);
#pragma unroll
    for (int j = 0; j < D; ++j) Y[j] = m::fma(-b0[j], sq, ah[j]);
    RHS::diag_b(Y, pp, tk + h, bm);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const T drift = (a0[j] + a1[j]) * (T(0.5) * h);
      const T noise = (bp[j] + bm[j] + T(2) * b0[j]) * (T(0.25) * dW[j]);
      const T fit = (bp[j] - bm[j]) * (m::fma(dW[j], dW[j], -h) * q4);
      unew[j] = uu[j] + (drift + (noise + fit));
    }
  }
  template <class R = RHS>
  __device__ __forceinline__ typename std::enable_if<!DiagNoise<R>::value>::type siea_step(
      const T*, const T*, T, T, T, T, const T*, T*) {}

  __device__ __forceinline__ bool advance(const SolveArgs& a) {
    if (k >= nrun) return true;
    if (kSde) {
      const unsigned long long stream = (unsigned long long)(a.index_offset + idx);
      T z[kPC * kCalls];
      if (kCalls == 1) {
        Normals<T>::draw(Philox::call(a.seed, stream, (unsigned long long)(unsigned(k) / unsigned(kSub))), z);
        if (k + kSub < n && k + kSub <= nrun) {  // all kSub steps run, none is the last
#pragma unroll
          for (int sub = 0; sub < kSub; ++sub) one_step<true>(a, z + sub * kNW);
        } else {
#pragma unroll
          for (int sub = 0; sub < kSub; ++sub)
            if (k < nrun) one_step(a, z + sub * kNW);
        }
      } else {
#pragma unroll
        for (int c = 0; c < kCalls; ++c)
          Normals<T>::draw(Philox::call(a.seed, stream, (unsigned long long)k * kCalls + c),
                           z + c * kPC);
        one_step(a, z);
      }
    } else {
      one_step(a, nullptr);
    }
    return k >= nrun;
  }

  __device__ __forceinline__ void finish(const SolveArgs& a) {
    signed char st = ENS_TRAJ_OK;
    bool fin = true;
#pragma unroll
    for (int j = 0; j < D; ++j) fin = fin && M<T>::finite(u[j]);
    if (nrun < n) st = ENS_TRAJ_MAXITERS;
    else if (!fin) st = ENS_TRAJ_NONFINITE;
    if (a.n_save == 0) write_slot<RHS, T>(a, idx, 0, u);
    for (; si < a.n_save; ++si) write_nan_slot<RHS, T>(a, idx, si);
    // f evaluations: Tsit5 1 + 6 per step (FSAL), RK4 4, Euler-Maruyama 1, SIEA 2 (drift at
    // X and at Ybar)
    const int fev = METH == METH_FIX_TSIT5 ? int(1 + 6 * k)
                    : METH == METH_FIX_RK4 ? int(4 * k)
                    : METH == METH_FIX_SIEA ? int(2 * k) : int(k);
    write_stats(a, idx, st, int(k), 0, fev);
  }

  // expected work: the number of fixed steps
  static __device__ __forceinline__ float cost_key(const SolveArgs& a, long long i, void*) {
    const double t0 = double(ldg<T>(a.tspan, in_idx(a.layout, i, 0, a.N, 2)));
    const double tf = double(ldg<T>(a.tspan, in_idx(a.layout, i, 1, a.N, 2)));
    return float((tf - t0) / a.dt);
  }
};

// ------------------------------------------------------------------------------------------
// schedules
__device__ __forceinline__ long long queue_next(unsigned long long* q) {
  const unsigned mask = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  const int rank = __popc(mask & ((1u << lane) - 1u));
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(q, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return (long long)(base + (unsigned long long)rank);
}

template <class I>
__global__ void k_direct(const SolveArgs a) {
  if constexpr (I::kSmemSaves)
    if (a.n_save > 0) load_save_times<typename I::Real>(a);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += stride) {
    I s;
    s.init(i, a);
    while (!s.advance(a)) {
    }
    s.finish(a);
  }
}

// ------------------------------------------------------------------------------------------
// Longest-expected-first ordering: a counting sort of log2 cost keys (32 buckets per octave).
// Pass 1 (a grid striding over all trajectories) computes each key's bucket and adds each
// block's histogram into the bucket totals.  Pass 2: block b of G owns trajectories
// [b*C, min((b+1)*C, N)); every block scans the 1024 totals itself (bucket starts), reserves
// one contiguous range per (block, bucket) with a single atomic on that bucket's fill cursor
// and scatters with shared-memory atomics.  (Order inside a bucket is arbitrary: the
// result of every trajectory does not depend on the order.)
__device__ __forceinline__ int cost_bucket(float key) {
  int b = (int)(log2f(fmaxf(key, 1.f)) * 32.f);  // NaN keys land in the cheapest bucket
  b = b < 0 ? 0 : (b > kCostBuckets - 1 ? kCostBuckets - 1 : b);
  return kCostBuckets - 1 - b;  // ascending bucket = descending cost
}

template <class I>
__global__ void k_cost_keys(const SolveArgs a, unsigned short* bucket, unsigned int* tot,
                            void* h0c) {
  __shared__ unsigned int sh[kCostBuckets];
  for (int b = threadIdx.x; b < kCostBuckets; b += blockDim.x) sh[b] = 0u;
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.N;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = cost_bucket(I::cost_key(a, i, h0c));
    bucket[i] = (unsigned short)b;
    atomicAdd(&sh[b], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kCostBuckets; b += blockDim.x)
    if (sh[b]) atomicAdd(&tot[b], sh[b]);
}

// the keys themselves (the work estimate that balances shards across ranks)
template <class I>
__global__ void k_cost_values(const SolveArgs a, float* keys) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.N;
       i += (long long)gridDim.x * blockDim.x)
    keys[i] = I::cost_key(a, i, nullptr);
}


// Persistent schedule.  Every lane of a warp stays in the loop until the whole warp is done,
// so warp-wide votes are safe.  A lane that finishes its trajectory writes it out and idles;
// once at least a.refill_min lanes of the warp are idle (or all are), the idle lanes fetch
// the next indices together (one warp-aggregated atomic) and initialise in one divergent
// pass instead of one pass per finishing lane.  The loop returns when the queue is drained
// and every lane of the warp is done (no block-wide synchronisation inside, so a kernel can
// run several solves' loops one after another per warp); with a.slots it adds the lane slots
// it issued (iterations x 32 x TPT), the denominator of the lane efficiency.
__device__ __forceinline__ void count_slots(unsigned long long* slots, unsigned long long n) {
  if (slots && (threadIdx.x & 31) == 0) atomicAdd(slots, n * 32ull);
}

template <class I, int TPT>
__device__ __forceinline__ void persistent_loop(const SolveArgs& a) {
  unsigned iters = 0;  // loop iterations of this warp
  I s[TPT];
  bool act[TPT];
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    const long long i = queue_next(a.queue);
    act[q] = i < a.N;
    if (act[q]) s[q].init(a.order ? (long long)__ldg(a.order + i) : i, a);
  }
  bool drained = __any_sync(0xffffffffu, !act[TPT - 1]);  // warp-uniform
  for (;;) {
    ++iters;
    unsigned busy = 0u;
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      if (act[q] && s[q].advance(a)) {
        s[q].finish(a);
        act[q] = false;
      }
      busy |= __ballot_sync(0xffffffffu, act[q]);
    }
    if (drained) {
      if (busy == 0u) break;
      continue;
    }
    if constexpr (TPT == 1) {
      const unsigned idle = __ballot_sync(0xffffffffu, !act[0]);
      if (__popc(idle) >= a.refill_min) {
        bool got = true;
        if (!act[0]) {
          const long long i = queue_next(a.queue);
          act[0] = i < a.N;
          got = act[0];
          if (act[0]) s[0].init(a.order ? (long long)__ldg(a.order + i) : i, a);
        }
        drained = drained || __any_sync(0xffffffffu, !got);
      }
    } else {
      // one refill pass over all slots: once the warp's 32 x TPT slots hold refill_min idle
      // ones, every thread with an idle slot fills its first idle one, so the warp runs the
      // initialisation once for all slot indices (the new state is copied into its slot by
      // selects, never through an indexed array)
      int nidle = 0;
#pragma unroll
      for (int q = 0; q < TPT; ++q) nidle += __popc(__ballot_sync(0xffffffffu, !act[q]));
      if (nidle >= a.refill_min) {
        bool got = true;
        int qf = -1;
#pragma unroll
        for (int q = TPT - 1; q >= 0; --q) qf = act[q] ? qf : q;
        if (qf >= 0) {
          const long long i = queue_next(a.queue);
          got = i < a.N;
          if (got) {
            I t;
            t.init(a.order ? (long long)__ldg(a.order + i) : i, a);
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
              if (q == qf) {
                s[q] = t;
                act[q] = true;
              }
            }
          }
        }
        drained = drained || __any_sync(0xffffffffu, !got);
      }
    }
  }
  count_slots(a.slots, (unsigned long long)iters * TPT * I::kStepsPerAdvance);
}

template <class I, int TPT>
__global__ void k_persistent(const SolveArgs a) {
  if constexpr (I::kSmemSaves)
    if (a.n_save > 0) load_save_times<typename I::Real>(a);
  persistent_loop<I, TPT>(a);
}

}  // namespace ens
