// ens_pair.cuh -- two trajectories per thread in lockstep on the paired FP32 instructions.
//
// sm_100-class GPUs issue FFMA2 / FADD2 / FMUL2: one instruction applies the same FP32 operation
// to the two halves of a register pair, rounding each exactly like the scalar instruction.  The
// adaptive Tsit5 solve is issue-bound (the FMA pipe is ~60 % busy when every issue slot is
// used), so a thread that advances two trajectories side by side -- lane 0 and lane 1 of
// float2 registers -- does the stage combinations, the right-hand sides, the error estimate
// and the norm with half the instructions.  Every lane performs exactly the operations of the
// scalar integrator, in the same order, so each trajectory's result is bit-identical to the
// one-trajectory-per-thread kernel.  Controller decisions, selects and the MUFU exponentials
// stay per lane.  Used for FP32 adaptive Tsit5 on autonomous models without save times (the
// persistent schedule with two trajectories per thread); initialisation and output reuse the
// scalar integrator.
#pragma once

#include "ens_kernels.cuh"

namespace ens {

__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float lane(float2 v, int k) { return k ? v.y : v.x; }
__device__ __forceinline__ void set_lane(float2& v, int k, float x) {
  v.x = k ? v.x : x;
  v.y = k ? x : v.y;
}

// Right-hand side on a pair of states.  Generic: the scalar f on each lane; Lorenz: the same
// association as Lorenz<float>::f with paired instructions.
template <class RHS>
struct Rhs2 {
  static constexpr int D = RHS::D, P = RHS::P;
  static __device__ __forceinline__ void f(const float2* u, const float2* p, float2* du) {
    float ux[D], uy[D], px[P], py[P], dx[D], dy[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      ux[j] = u[j].x;
      uy[j] = u[j].y;
    }
#pragma unroll
    for (int j = 0; j < P; ++j) {
      px[j] = p[j].x;
      py[j] = p[j].y;
    }
    RHS::f(ux, px, 0.f, dx);
    RHS::f(uy, py, 0.f, dy);
#pragma unroll
    for (int j = 0; j < D; ++j) du[j] = make_float2(dx[j], dy[j]);
  }
};
template <>
struct Rhs2<Lorenz<float>> {
  static __device__ __forceinline__ void f(const float2* u, const float2* p, float2* du) {
    du[0] = mul2(p[0], sub2(u[1], u[0]));               // sigma (y2 - y1)
    du[1] = fma2(u[0], sub2(p[1], u[2]), neg2(u[1]));   // y1 (rho - y3) - y2
    du[2] = fma2(u[0], u[1], neg2(mul2(p[2], u[2])));   // y1 y2 - beta y3
  }
};

// One Tsit5 step on a pair (tsit5_step, same association); es only with WANT_ERR.
template <class RHS, bool WANT_ERR = true>
__device__ __forceinline__ void tsit5_step2(const float2* u, const float2* p, float2 h,
                                            const float2* k1, float2* unew, float2* es,
                                            float2* k7) {
  constexpr int D = RHS::D;
  typedef Rhs2<RHS> F;
  float2 U[D], k2[D], k3[D], k4[D], k5[D], k6[D];
#pragma unroll
  for (int j = 0; j < D; ++j) U[j] = fma2(h, mul2(bc2(float(Ts5::a21)), k1[j]), u[j]);
  F::f(U, p, k2);
#pragma unroll
  for (int j = 0; j < D; ++j)
    U[j] = fma2(h, fma2(bc2(float(Ts5::a32)), k2[j], mul2(bc2(float(Ts5::a31)), k1[j])), u[j]);
  F::f(U, p, k3);
#pragma unroll
  for (int j = 0; j < D; ++j)
    U[j] = fma2(h,
                fma2(bc2(float(Ts5::a43)), k3[j],
                     fma2(bc2(float(Ts5::a42)), k2[j], mul2(bc2(float(Ts5::a41)), k1[j]))),
                u[j]);
  F::f(U, p, k4);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    float2 s = mul2(bc2(float(Ts5::a51)), k1[j]);
    s = fma2(bc2(float(Ts5::a52)), k2[j], s);
    s = fma2(bc2(float(Ts5::a53)), k3[j], s);
    s = fma2(bc2(float(Ts5::a54)), k4[j], s);
    U[j] = fma2(h, s, u[j]);
  }
  F::f(U, p, k5);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    float2 s = mul2(bc2(float(Ts5::a61)), k1[j]);
    s = fma2(bc2(float(Ts5::a62)), k2[j], s);
    s = fma2(bc2(float(Ts5::a63)), k3[j], s);
    s = fma2(bc2(float(Ts5::a64)), k4[j], s);
    s = fma2(bc2(float(Ts5::a65)), k5[j], s);
    U[j] = fma2(h, s, u[j]);
  }
  F::f(U, p, k6);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    float2 s = mul2(bc2(float(Ts5::a71)), k1[j]);
    s = fma2(bc2(float(Ts5::a72)), k2[j], s);
    s = fma2(bc2(float(Ts5::a73)), k3[j], s);
    s = fma2(bc2(float(Ts5::a74)), k4[j], s);
    s = fma2(bc2(float(Ts5::a75)), k5[j], s);
    s = fma2(bc2(float(Ts5::a76)), k6[j], s);
    unew[j] = fma2(h, s, u[j]);
  }
  F::f(unew, p, k7);
  if constexpr (WANT_ERR) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float2 s = mul2(bc2(float(Ts5::bt1)), k1[j]);
      s = fma2(bc2(float(Ts5::bt2)), k2[j], s);
      s = fma2(bc2(float(Ts5::bt3)), k3[j], s);
      s = fma2(bc2(float(Ts5::bt4)), k4[j], s);
      s = fma2(bc2(float(Ts5::bt5)), k5[j], s);
      s = fma2(bc2(float(Ts5::bt6)), k6[j], s);
      s = fma2(bc2(float(Ts5::bt7)), k7[j], s);
      es[j] = s;
    }
  }
}

// One classical RK4 step on a pair (rk4_step, same association; the factor 2 is exact, so
// its product rounds alike contracted or not).
template <class RHS>
__device__ __forceinline__ void rk4_step2(const float2* u, const float2* p, float2 h,
                                          float2* unew) {
  constexpr int D = RHS::D;
  typedef Rhs2<RHS> F;
  float2 k1[D], k2[D], k3[D], k4[D], U[D];
  const float2 hh = mul2(bc2(0.5f), h);
  F::f(u, p, k1);
#pragma unroll
  for (int j = 0; j < D; ++j) U[j] = fma2(hh, k1[j], u[j]);
  F::f(U, p, k2);
#pragma unroll
  for (int j = 0; j < D; ++j) U[j] = fma2(hh, k2[j], u[j]);
  F::f(U, p, k3);
#pragma unroll
  for (int j = 0; j < D; ++j) U[j] = fma2(h, k3[j], u[j]);
  F::f(U, p, k4);
  const float2 h6 = mul2(h, bc2(float(1.0 / 6.0)));
#pragma unroll
  for (int j = 0; j < D; ++j)
    unew[j] = fma2(h6, fma2(bc2(2.f), add2(k2[j], k3[j]), add2(k1[j], k4[j])), u[j]);
}

// Two adaptive Tsit5 trajectories (FP32, no save times) advanced in lockstep.
template <class RHS>
struct AdaptivePair {
  static_assert(RHS::autonomous, "the paired integrator passes no time to f");
  static constexpr int D = RHS::D, P = RHS::P;
  typedef Adaptive<RHS, float, METH_TSIT5> Scalar;

  float2 u[D], fk[D], p[P];
  float2 hi, lo;   // compensated time (Neumaier pair), per lane
  float2 stop, thr, h;
  float2 lq;
  int attempts[2], rejected[2], fev0[2], st[2];
  long long idx[2];

  // k may be a run-time lane (the refill pass serves lane 0 of some threads and lane 1 of
  // others at once): every write is then a select, never an indexed register array
  __device__ __forceinline__ static void set2(int (&v)[2], int k, int x) {
    v[0] = k ? v[0] : x;
    v[1] = k ? x : v[1];
  }
  __device__ __forceinline__ void init(int k, long long i, const SolveArgs& a) {
    Scalar s;
    s.template init<false>(i, a);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      set_lane(u[j], k, s.u[j]);
      set_lane(fk[j], k, s.fk[j]);
    }
#pragma unroll
    for (int j = 0; j < P; ++j) set_lane(p[j], k, s.p[j]);
    set_lane(hi, k, s.t.hi);
    set_lane(lo, k, s.t.lo);
    set_lane(stop, k, s.stop);
    set_lane(thr, k, s.stop_thr);
    set_lane(h, k, s.h);
    set_lane(lq, k, s.lq);
    set2(attempts, k, s.attempts);
    set2(rejected, k, s.rejected);
    set2(fev0, k, s.fev0);
    set2(st, k, s.st);
    idx[0] = k ? idx[0] : s.idx;
    idx[1] = k ? s.idx : idx[1];
  }

  __device__ __forceinline__ void finish(int k, const SolveArgs& a) {
    Scalar s;
#pragma unroll
    for (int j = 0; j < D; ++j) s.u[j] = lane(u[j], k);
    s.idx = idx[k];
    s.si = 0;
    s.st = st[k];
    s.attempts = attempts[k];
    s.rejected = rejected[k];
    s.fev0 = fev0[k];
    s.nev = 0;  // the paired kernel serves models without events
    s.template finish<false>(a);
  }

  // One attempt for each live lane; returns the mask of lanes that finished (arrived at tf
  // or failed).  Finished and idle lanes keep their state.
  __device__ __forceinline__ unsigned advance(const SolveArgs& a, bool live0, bool live1) {
    bool live[2] = {live0, live1};
    unsigned done = 0u;
    const float2 rem = sub2(sub2(stop, hi), lo);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (live[k] && lane(rem, k) <= lane(thr, k)) {  // arrived at tf: t = tf
        set_lane(hi, k, lane(stop, k));
        set_lane(lo, k, 0.f);
        done |= 1u << k;
        live[k] = false;
      }
    }
    if (!live[0] && !live[1]) return done;
    bool last[2];
    float2 hs;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      last[k] = lane(h, k) >= lane(rem, k);
      set_lane(hs, k, last[k] ? lane(rem, k) : lane(h, k));
    }
    const float2 tnow = add2(hi, lo);
    float2 unew[D], es[D], fnew[D];
    tsit5_step2<RHS>(u, p, hs, fk, unew, es, fnew);
    const float atol = a.abstol_f, rtol = a.reltol_f;
    float2 r2 = bc2(0.f);
    float2 he[D], sc[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      he[j] = mul2(hs, es[j]);
      sc[j] = fma2(bc2(rtol),
                   make_float2(fmaxf(fabsf(u[j].x), fabsf(unew[j].x)),
                               fmaxf(fabsf(u[j].y), fabsf(unew[j].y))),
                   bc2(atol));
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const float2 r = make_float2(__fdividef(he[j].x, sc[j].x), __fdividef(he[j].y, sc[j].y));
      r2 = fma2(r, r, r2);
    }
    const float2 q2 = mul2(r2, bc2(1.f / float(D)));
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (!live[k]) continue;
      bool fin = true;
#pragma unroll
      for (int j = 0; j < D; ++j) fin = fin && isfinite(lane(unew[j], k));
      const float qk = lane(q2, k);
      const float hk = lane(hs, k);
      const bool capped = attempts[k] >= a.maxiters_i;
      const bool tiny = hk < float(M<float>::dtmin_factor) * fmaxf(1.f, fabsf(lane(tnow, k)));
      if (capped || tiny || !fin || isnan(qk)) {
        st[k] = capped ? ENS_TRAJ_MAXITERS : (tiny ? ENS_TRAJ_DT_MIN : ENS_TRAJ_NONFINITE);
        attempts[k] += (capped || tiny) ? 0 : 1;
        done |= 1u << k;
        continue;
      }
      ++attempts[k];
      const bool acc = qk <= 1.f;
      const float L = lg2_approx(fmaxf(qk, 1e-20f));
      const float e = acc ? __fmaf_rn(-0.35f / 5.f, L, (0.4f / 5.f) * lane(lq, k))
                          : (-0.5f / 5.f) * L;
      const float fac = fminf(acc ? 10.f : 1.f, fmaxf(0.2f, float(kEta) * ex2_approx(e)));
#pragma unroll
      for (int j = 0; j < D; ++j) {
        set_lane(u[j], k, acc ? lane(unew[j], k) : lane(u[j], k));
        set_lane(fk[j], k, acc ? lane(fnew[j], k) : lane(fk[j], k));
      }
      Clock<float> t;
      t.hi = lane(hi, k);
      t.lo = lane(lo, k);
      t.add(acc ? hk : 0.f);
      t.snap(acc && last[k], lane(stop, k));
      set_lane(hi, k, t.hi);
      set_lane(lo, k, t.lo);
      set_lane(lq, k, acc ? fmaxf(0.5f * L, kLog2QoldInit) : lane(lq, k));
      rejected[k] += acc ? 0 : 1;
      set_lane(h, k, hk * fac);
    }
    return done;
  }
};

// Persistent schedule with one AdaptivePair per thread: the refill logic of persistent_loop
// with two slots, the slots being the two lanes.
template <class RHS>
__device__ __forceinline__ void persistent_pair_loop(const SolveArgs& a) {
  unsigned iters = 0;  // loop iterations of this warp
  AdaptivePair<RHS> s;
  bool act[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const long long i = queue_next(a.queue);
    act[q] = i < a.N;
    if (act[q]) s.init(q, a.order ? (long long)__ldg(a.order + i) : i, a);
  }
  bool drained = __any_sync(0xffffffffu, !act[1]);  // warp-uniform
  for (;;) {
    ++iters;
    if (act[0] || act[1]) {
      const unsigned done = s.advance(a, act[0], act[1]);
#pragma unroll
      for (int q = 0; q < 2; ++q)
        if (done & (1u << q)) {
          s.finish(q, a);
          act[q] = false;
        }
    }
    const unsigned busy = __ballot_sync(0xffffffffu, act[0] || act[1]);
    if (drained) {
      if (busy == 0u) break;
      continue;
    }
    // one refill pass over both lanes: once the warp's 64 slots hold refill_min idle ones,
    // every thread with an idle slot fills one of them (lane 0 first), so the warp runs the
    // initialisation once for both lanes' idle slots; a thread with both idle fills the
    // other at a later pass
    const unsigned idle0 = __ballot_sync(0xffffffffu, !act[0]);
    const unsigned idle1 = __ballot_sync(0xffffffffu, !act[1]);
    if (__popc(idle0) + __popc(idle1) >= a.refill_min) {
      bool got = true;
      if (!act[0] || !act[1]) {
        const int q = act[0] ? 1 : 0;
        const long long i = queue_next(a.queue);
        got = i < a.N;
        if (got) {
          s.init(q, a.order ? (long long)__ldg(a.order + i) : i, a);
          act[0] = act[0] || q == 0;
          act[1] = act[1] || q == 1;
        }
      }
      drained = drained || __any_sync(0xffffffffu, !got);
    }
  }
  count_slots(a.slots, (unsigned long long)iters * 2);
}

template <class RHS>
__global__ void k_persistent_pair(const SolveArgs a) {
  persistent_pair_loop<RHS>(a);
}

// Fixed-step Tsit5 or RK4 on two trajectories per thread (FP32, final state only, the direct
// schedule): the two lanes take the scalar integrator's steps side by side, the last step of
// each lane shortened to land on its tf as in Fixed::one_step; once one lane's steps are
// done it keeps its state (selects) while the other finishes.  Initialisation and output are
// the scalar integrator's, so results, status and counters equal the one-per-thread kernel's
// bit for bit.  With equal step counts (one tspan for the whole ensemble) no lane idles.
template <class RHS, int METH>
__global__ void k_direct_pair(const SolveArgs a) {
  static_assert(RHS::autonomous, "the paired integrator passes no time to f");
  static_assert(METH == METH_FIX_TSIT5 || METH == METH_FIX_RK4, "Tsit5 or RK4");
  typedef Fixed<RHS, float, METH> Scalar;
  constexpr int D = RHS::D, P = RHS::P;
  const long long stride = 2LL * gridDim.x * blockDim.x;
  for (long long i0 = 2LL * ((long long)blockIdx.x * blockDim.x + threadIdx.x); i0 < a.N;
       i0 += stride) {
    const bool two = i0 + 1 < a.N;
    Scalar s0, s1;
    s0.init(i0, a);
    s1.init(two ? i0 + 1 : i0, a);  // a lone last trajectory: lane 1 repeats it, unwritten
    float2 u[D], fk[D], p[P];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      u[j] = make_float2(s0.u[j], s1.u[j]);
      fk[j] = make_float2(s0.fk[j], s1.fk[j]);
    }
#pragma unroll
    for (int j = 0; j < P; ++j) p[j] = make_float2(s0.p[j], s1.p[j]);
    const int m0 = s0.nrun, m1 = two ? s1.nrun : 0;
    const int last0 = s0.n - 1, last1 = s1.n - 1;
    const float hr = s0.h_reg, hl0 = s0.h_last, hl1 = s1.h_last;
    const int mlo = m0 < m1 ? m0 : m1, mhi = m0 < m1 ? m1 : m0;
    // steps before either lane's last one take the regular step on both lanes: no per-step
    // choice of h (and the step's constant multiples of h hoisted out of the loop)
    const int lmin = last0 < last1 ? last0 : last1;
    const int mreg = lmin < mlo ? (lmin > 0 ? lmin : 0) : mlo;
    const float2 hreg = bc2(hr);
    int k = 0;
    for (; k < mreg; ++k) {
      float2 unew[D], k7[D];
      if constexpr (METH == METH_FIX_TSIT5)
        tsit5_step2<RHS, false>(u, p, hreg, fk, unew, nullptr, k7);
      else
        rk4_step2<RHS>(u, p, hreg, unew);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        u[j] = unew[j];
        if constexpr (METH == METH_FIX_TSIT5) fk[j] = k7[j];
      }
    }
    for (; k < mlo; ++k) {  // both lanes step
      const float2 h = make_float2(k == last0 ? hl0 : hr, k == last1 ? hl1 : hr);
      float2 unew[D], k7[D];
      if constexpr (METH == METH_FIX_TSIT5)
        tsit5_step2<RHS, false>(u, p, h, fk, unew, nullptr, k7);
      else
        rk4_step2<RHS>(u, p, h, unew);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        u[j] = unew[j];
        if constexpr (METH == METH_FIX_TSIT5) fk[j] = k7[j];
      }
    }
    for (; k < mhi; ++k) {  // one lane steps, the other keeps its final state
      const bool l0 = k < m0, l1 = k < m1;
      const float2 h = make_float2(k == last0 ? hl0 : hr, k == last1 ? hl1 : hr);
      float2 unew[D], k7[D];
      if constexpr (METH == METH_FIX_TSIT5)
        tsit5_step2<RHS, false>(u, p, h, fk, unew, nullptr, k7);
      else
        rk4_step2<RHS>(u, p, h, unew);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        u[j] = make_float2(l0 ? unew[j].x : u[j].x, l1 ? unew[j].y : u[j].y);
        if constexpr (METH == METH_FIX_TSIT5)
          fk[j] = make_float2(l0 ? k7[j].x : fk[j].x, l1 ? k7[j].y : fk[j].y);
      }
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
      s0.u[j] = u[j].x;
      s1.u[j] = u[j].y;
    }
    s0.k = m0;
    s0.finish(a);
    if (two) {
      s1.k = m1;
      s1.finish(a);
    }
  }
}

}  // namespace ens
