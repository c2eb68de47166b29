// adjoint.cuh -- discrete adjoint of the fixed-step explicit Runge-Kutta map, one thread per
// trajectory, with checkpointing.
//
// The paper differentiates through its GPU solvers by automatic differentiation (Sec. 6.5:
// the solvers are compatible with forward- and reverse-mode AD).  Here the reverse mode is
// written out by hand for the step map of Sec. 3.1,
//     U_i = u_n + h sum_{j<i} a_ij k_j,   k_i = f(U_i, p),   u_{n+1} = u_n + h sum_i b_i k_i,
// whose transpose, with lambda = dL/du_{n+1}, is
//     kbar_i = h b_i lambda + h sum_{l>i} a_li Ubar_l,   Ubar_i = f_u(U_i)^T kbar_i,
//     pbar  += f_p(U_i)^T kbar_i,                        dL/du_n = lambda + sum_i Ubar_i,
// taken for i = s, ..., 1 (kbar_i is complete once every later stage has been processed).
//
// Memory plan: the forward pass stores u every K steps (checkpoints [C][D][N]); the reverse
// pass walks the segments backwards, replays each one from its checkpoint while storing the
// stage inputs U_1..U_s of every step ([K][s][D][N], coalesced across trajectories) and then
// runs the transposed steps over the stored stages, so no stage is evaluated twice in the
// reverse pass.  (FP64 runs at 1/72 of the FP32 rate on GB300 while HBM is plentiful: storing
// the s stage inputs costs s*D*8 bytes per step, recomputing them costs a whole forward step.)
#pragma once

#include "ens_kernels.cuh"

namespace ens {

// Tsit5's propagating map uses stages 1..6 (its seventh, FSAL stage has b_7 = 0); the
// coefficients are those of the solver (Tsitouras 2011), b_i = a_7i.
struct TabTsit5 {
  static constexpr int S = 6;
  static __device__ __forceinline__ constexpr double c(int i) {
    return i == 0 ? 0.0 : i == 1 ? Ts5::c2 : i == 2 ? Ts5::c3 : i == 3 ? Ts5::c4
         : i == 4 ? Ts5::c5 : 1.0;
  }
  static __device__ __forceinline__ constexpr double a(int i, int j) {
    return i == 1 ? Ts5::a21
         : i == 2 ? (j == 0 ? Ts5::a31 : Ts5::a32)
         : i == 3 ? (j == 0 ? Ts5::a41 : j == 1 ? Ts5::a42 : Ts5::a43)
         : i == 4 ? (j == 0 ? Ts5::a51 : j == 1 ? Ts5::a52 : j == 2 ? Ts5::a53 : Ts5::a54)
         : (j == 0 ? Ts5::a61 : j == 1 ? Ts5::a62 : j == 2 ? Ts5::a63 : j == 3 ? Ts5::a64
                                                                                 : Ts5::a65);
  }
  static __device__ __forceinline__ constexpr double b(int i) {
    return i == 0 ? Ts5::a71 : i == 1 ? Ts5::a72 : i == 2 ? Ts5::a73 : i == 3 ? Ts5::a74
         : i == 4 ? Ts5::a75 : Ts5::a76;
  }
};

// Classic RK4: c = (0, 1/2, 1/2, 1), a_21 = a_32 = 1/2, a_43 = 1, b = (1, 2, 2, 1)/6.
struct TabRK4 {
  static constexpr int S = 4;
  static __device__ __forceinline__ constexpr double c(int i) {
    return i == 0 ? 0.0 : i == 3 ? 1.0 : 0.5;
  }
  static __device__ __forceinline__ constexpr double a(int i, int j) {
    return (j != i - 1) ? 0.0 : (i == 3 ? 1.0 : 0.5);
  }
  static __device__ __forceinline__ constexpr double b(int i) {
    return (i == 0 || i == 3) ? 1.0 / 6.0 : 1.0 / 3.0;
  }
};


__device__ __forceinline__ long long adj_idx(int layout, long long i, int k, long long N, int w) {
  return layout == ENS_LAYOUT_SOA ? (long long)k * N + i : i * w + k;
}

// Number of fixed steps n = ceil((tf - t0)/dt - 1e-12) and the last step h_last =
// tf - (t0 + (n-1) dt), the same arithmetic as the forward solver.
__device__ __forceinline__ long long adj_steps(double t0, double tf, double dt, double* h_last) {
  long long n = (tf > t0) ? (long long)ceil((tf - t0) / dt - 1e-12) : 0;
  if (n < 0) n = 0;
  *h_last = n > 0 ? tf - (t0 + double(n - 1) * dt) : 0.0;
  return n;
}

// One explicit RK step in tableau form; stage sums associate exactly like tsit5_step
// (s = a_i1 k_1, then fused multiply-adds in j, U = fma(h, s, u)).  With STORE, the stage
// inputs U_1..U_s go to seg[(kk*S + i)*D + j][tid] (stride N).
template <class RHS, class T, class TAB, bool STORE>
__device__ __forceinline__ void rk_tab_step(T* u, const T* p, T t, T h, T* seg, long long kk,
                                            long long tid, long long N) {
  constexpr int D = RHS::D, S = TAB::S;
  typedef M<T> m;
  T k[S][D], U[D];
#pragma unroll
  for (int i = 0; i < S; ++i) {
    if (i == 0) {
#pragma unroll
      for (int j = 0; j < D; ++j) U[j] = u[j];
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        T s = T(0);
        bool first = true;  // folded at compile time: the sum starts at the first nonzero a_il
#pragma unroll
        for (int l = 0; l < i; ++l)
          if (TAB::a(i, l) != 0.0) {
            s = first ? T(TAB::a(i, l)) * k[l][j] : m::fma(T(TAB::a(i, l)), k[l][j], s);
            first = false;
          }
        U[j] = m::fma(h, s, u[j]);
      }
    }
    if (STORE) {
#pragma unroll
      for (int j = 0; j < D; ++j) seg[((kk * S + i) * D + j) * N + tid] = U[j];
    }
    RHS::f(U, p, t + T(TAB::c(i)) * h, k[i]);
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    T s = T(TAB::b(0)) * k[0][j];
#pragma unroll
    for (int l = 1; l < S; ++l) s = m::fma(T(TAB::b(l)), k[l][j], s);
    u[j] = m::fma(h, s, u[j]);
  }
}

// The transposed step: lam = dL/du_{n+1} in, dL/du_n out; pb accumulates dL/dp.
template <class RHS, class T, class TAB>
__device__ __forceinline__ void rk_tab_step_adjoint(T* lam, T* pb, const T* p, T t, T h,
                                                    const T* seg, long long kk, long long tid,
                                                    long long N) {
  constexpr int D = RHS::D, P = RHS::P, S = TAB::S;
  typedef M<T> m;
  T kb[S][D], ub[D], lh[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    lh[j] = h * lam[j];
    ub[j] = lam[j];
  }
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) kb[i][j] = T(TAB::b(i)) * lh[j];
#pragma unroll
  for (int i = S - 1; i >= 0; --i) {
    T U[D], Ub[D], pg[P];
#pragma unroll
    for (int j = 0; j < D; ++j) U[j] = seg[((kk * S + i) * D + j) * N + tid];
    const T ti = t + T(TAB::c(i)) * h;
    RHS::vjp_u(U, p, ti, kb[i], Ub);
    RHS::vjp_p(U, p, ti, kb[i], pg);
#pragma unroll
    for (int q = 0; q < P; ++q) pb[q] += pg[q];
#pragma unroll
    for (int j = 0; j < D; ++j) ub[j] += Ub[j];
    if (i > 0) {
      T Uh[D];
#pragma unroll
      for (int j = 0; j < D; ++j) Uh[j] = h * Ub[j];
#pragma unroll
      for (int l = 0; l < i; ++l)
        if (TAB::a(i, l) != 0.0) {
#pragma unroll
          for (int j = 0; j < D; ++j) kb[l][j] = m::fma(T(TAB::a(i, l)), Uh[j], kb[l][j]);
        }
    }
  }
#pragma unroll
  for (int j = 0; j < D; ++j) lam[j] = ub[j];
}

template <class RHS, class T>
__device__ __forceinline__ void adj_load(const AdjArgs& a, long long i, T* p, T* u, double* t0,
                                         double* tf) {
  constexpr int D = RHS::D, P = RHS::P;
#pragma unroll
  for (int k = 0; k < P; ++k)
    p[k] = __ldg(static_cast<const T*>(a.params) + adj_idx(a.layout, i, k, a.N, P));
#pragma unroll
  for (int k = 0; k < D; ++k)
    u[k] = __ldg(static_cast<const T*>(a.u0) + adj_idx(a.layout, i, k, a.N, D));
  *t0 = double(__ldg(static_cast<const T*>(a.tspan) + adj_idx(a.layout, i, 0, a.N, 2)));
  *tf = double(__ldg(static_cast<const T*>(a.tspan) + adj_idx(a.layout, i, 1, a.N, 2)));
}

// Forward pass with checkpoints: ckpt[c][j][i] = u_{cK}, j < D, for c < ceil(n/K); out = u_n.
template <class RHS, class T, class TAB>
__global__ void k_adj_forward(const AdjArgs a) {
  constexpr int D = RHS::D, P = RHS::P;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  T p[P], u[D];
  double t0, tf, hl;
  adj_load<RHS, T>(a, i, p, u, &t0, &tf);
  const long long n = adj_steps(t0, tf, a.dt, &hl);
  const bool fits = n <= a.max_steps;
  T* ck = static_cast<T*>(a.ckpt);
  const T h = T(a.dt), h_last = T(hl), t0t = T(t0);
  if (fits) {
    for (long long k = 0; k < n; ++k) {
      if (k % a.K == 0) {
#pragma unroll
        for (int j = 0; j < D; ++j) ck[((k / a.K) * D + j) * a.N + i] = u[j];
      }
      const T tk = RHS::autonomous ? T(0) : t0t + T(k) * h;
      rk_tab_step<RHS, T, TAB, false>(u, p, tk, k == n - 1 ? h_last : h, nullptr, 0, i, a.N);
    }
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j) u[j] = nan_of<T>();
  }
  if (a.out) {
    T* o = static_cast<T*>(a.out);
#pragma unroll
    for (int j = 0; j < D; ++j) o[adj_idx(a.layout, i, j, a.N, D)] = u[j];
  }
  if (a.status) a.status[i] = fits ? ENS_TRAJ_OK : ENS_TRAJ_MAXITERS;
}

// Reverse pass over the checkpoints written by k_adj_forward (same arguments).
template <class RHS, class T, class TAB>
__global__ void k_adj_backward(const AdjArgs a) {
  constexpr int D = RHS::D, P = RHS::P;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  T p[P], u[D], lam[D], pb[P];
  double t0, tf, hl;
  adj_load<RHS, T>(a, i, p, u, &t0, &tf);
  const long long n = adj_steps(t0, tf, a.dt, &hl);
#pragma unroll
  for (int j = 0; j < D; ++j)
    lam[j] = __ldg(static_cast<const T*>(a.grad_out) + adj_idx(a.layout, i, j, a.N, D));
#pragma unroll
  for (int q = 0; q < P; ++q) pb[q] = T(0);
  const T h = T(a.dt), h_last = T(hl), t0t = T(t0);
  const T* ck = static_cast<const T*>(a.ckpt);
  T* seg = static_cast<T*>(a.seg);
  if (n <= a.max_steps) {
    const long long C = (n + a.K - 1) / a.K;
    for (long long c = C - 1; c >= 0; --c) {
      const long long k0 = c * a.K;
      const long long k1 = (k0 + a.K < n) ? k0 + a.K : n;
#pragma unroll
      for (int j = 0; j < D; ++j) u[j] = ck[(c * D + j) * a.N + i];
      for (long long k = k0; k < k1; ++k) {
        const T tk = RHS::autonomous ? T(0) : t0t + T(k) * h;
        rk_tab_step<RHS, T, TAB, true>(u, p, tk, k == n - 1 ? h_last : h, seg, k - k0, i, a.N);
      }
      for (long long k = k1 - 1; k >= k0; --k) {
        const T tk = RHS::autonomous ? T(0) : t0t + T(k) * h;
        rk_tab_step_adjoint<RHS, T, TAB>(lam, pb, p, tk, k == n - 1 ? h_last : h, seg, k - k0,
                                         i, a.N);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j) lam[j] = nan_of<T>();
#pragma unroll
    for (int q = 0; q < P; ++q) pb[q] = nan_of<T>();
  }
  T* gp = static_cast<T*>(a.grad_p);
  T* gu = static_cast<T*>(a.grad_u0);
#pragma unroll
  for (int q = 0; q < P; ++q) gp[adj_idx(a.layout, i, q, a.N, P)] = pb[q];
#pragma unroll
  for (int j = 0; j < D; ++j) gu[adj_idx(a.layout, i, j, a.N, D)] = lam[j];
}

}  // namespace ens
