// ens_device.cuh -- device-side building blocks of the ensemble solver (sm_103a).
//
// Everything here runs inside one thread and keeps its state in registers: the models'
// right-hand sides and Jacobians (Appendix: Lorenz, Robertson, linear SDE), the Tsit5 / RK4 /
// Rosenbrock23 / Euler-Maruyama steps (Sec. 3.1, 3.2.1, 3.3), the in-register LU of the
// Rosenbrock matrix (Sec. 5.1.3 batched LU, fused per thread) and Philox4x32-10.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

namespace ens {

// ------------------------------------------------------------------------------------------
// precision helpers
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <class T>
struct M;

template <>
struct M<float> {
  static __device__ __forceinline__ float fma(float a, float b, float c) {
    return __fmaf_rn(a, b, c);
  }
  static __device__ __forceinline__ float abs(float a) { return fabsf(a); }
  static __device__ __forceinline__ float max(float a, float b) { return fmaxf(a, b); }
  static __device__ __forceinline__ float min(float a, float b) { return fminf(a, b); }
  static __device__ __forceinline__ float sqrt(float a) { return sqrtf(a); }
  static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
  static __device__ __forceinline__ float pow(float a, float b) { return powf(a, b); }
  // approximate forms for heuristics (controller, starting step): MUFU ex2 / lg2
  static __device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float fast_pow(float a, float b) {
    return ex2_approx(b * lg2_approx(a));
  }
  // MUFU square root (sqrt.approx, about 1 ulp; subnormal inputs flush to 0)
  static __device__ __forceinline__ float fast_sqrt(float a) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
  }
  static __device__ __forceinline__ bool finite(float a) { return isfinite(a); }
  static constexpr double dtmin_factor = 1e-9;
};

template <>
struct M<double> {
  static __device__ __forceinline__ double fma(double a, double b, double c) {
    return __fma_rn(a, b, c);
  }
  static __device__ __forceinline__ double abs(double a) { return fabs(a); }
  static __device__ __forceinline__ double max(double a, double b) { return fmax(a, b); }
  static __device__ __forceinline__ double min(double a, double b) { return fmin(a, b); }
  static __device__ __forceinline__ double sqrt(double a) { return ::sqrt(a); }
  static __device__ __forceinline__ double rcp(double a) { return 1.0 / a; }
  static __device__ __forceinline__ double pow(double a, double b) { return ::pow(a, b); }
  static __device__ __forceinline__ double fast_div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double fast_pow(double a, double b) { return ::pow(a, b); }
  static __device__ __forceinline__ double fast_sqrt(double a) { return ::sqrt(a); }
  static __device__ __forceinline__ bool finite(double a) { return isfinite(a); }
  static constexpr double dtmin_factor = 1e-14;
};

// Structural nonzeros of a D x D matrix.
template <int D>
struct Pattern {
  bool nz[D][D];
};

// Calls f(std::integral_constant<int, i>) for i in [B, E), halving the range (shallow
// template recursion).
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (E - B == 1) {
    f(std::integral_constant<int, B>());
  } else if constexpr (E - B > 1) {
    constexpr int Mid = B + (E - B) / 2;
    static_for<B, Mid>(f);
    static_for<Mid, E>(f);
  }
}

// ------------------------------------------------------------------------------------------
// Models.  f = du/dt (drift for SDEs), jac = df/du (row-major D x D), vjp_u = (df/du)^T w,
// vjp_p = (df/dp)^T w.  SDE models (has_noise) have NW Wiener processes and
// sde(u, p, t, sq, z, a, b): the drift a(u) and the noise increment b_j = sum_m G_jm(u) sq z_m
// of one Euler-Maruyama step with sqrt(h) = sq and normals z[NW].  sde_only models have no
// Jacobian and take Euler-Maruyama only.

template <class T>
struct Lorenz {
  static constexpr int D = 3, P = 3, NW = 0;
  static constexpr bool autonomous = true, has_noise = false, sde_only = false, has_event = false;
  static constexpr bool stiff_only = false;
  static __device__ __forceinline__ void f(const T* u, const T* p, T, T* du) {
    du[0] = p[0] * (u[1] - u[0]);                  // sigma (y2 - y1)
    du[1] = M<T>::fma(u[0], p[1] - u[2], -u[1]);   // y1 (rho - y3) - y2
    du[2] = M<T>::fma(u[0], u[1], -(p[2] * u[2])); // y1 y2 - beta y3
  }
  static __device__ __forceinline__ void jac(const T* u, const T* p, T, T* J) {
    J[0] = -p[0]; J[1] = p[0]; J[2] = T(0);
    J[3] = p[1] - u[2]; J[4] = T(-1); J[5] = -u[0];
    J[6] = u[1]; J[7] = u[0]; J[8] = -p[2];
  }
  static __device__ __forceinline__ void vjp_u(const T* u, const T* p, T, const T* w, T* o) {
    o[0] = M<T>::fma(-p[0], w[0], M<T>::fma(p[1] - u[2], w[1], u[1] * w[2]));
    o[1] = M<T>::fma(p[0], w[0], M<T>::fma(u[0], w[2], -w[1]));
    o[2] = M<T>::fma(-u[0], w[1], -(p[2] * w[2]));
  }
  static __device__ __forceinline__ void vjp_p(const T* u, const T*, T, const T* w, T* o) {
    o[0] = (u[1] - u[0]) * w[0];
    o[1] = u[0] * w[1];
    o[2] = -u[2] * w[2];
  }
};

template <class T>
struct Robertson {
  static constexpr int D = 3, P = 3, NW = 0;
  static constexpr bool autonomous = true, has_noise = false, sde_only = false, has_event = false;
  static constexpr bool stiff_only = false;
  static __device__ __forceinline__ void f(const T* u, const T* p, T, T* du) {
    const T r1 = p[0] * u[0];           // k1 y1
    const T r2 = p[1] * u[1] * u[1];    // k2 y2^2
    const T r3 = p[2] * u[1] * u[2];    // k3 y2 y3
    du[0] = r3 - r1;
    du[1] = (r1 - r3) - r2;
    du[2] = r2;
  }
  static __device__ __forceinline__ void jac(const T* u, const T* p, T, T* J) {
    const T k3y3 = p[2] * u[2], k3y2 = p[2] * u[1], k2y2x2 = T(2) * p[1] * u[1];
    J[0] = -p[0]; J[1] = k3y3; J[2] = k3y2;
    J[3] = p[0]; J[4] = -k3y3 - k2y2x2; J[5] = -k3y2;
    J[6] = T(0); J[7] = k2y2x2; J[8] = T(0);
  }
  static __device__ __forceinline__ void vjp_u(const T* u, const T* p, T, const T* w, T* o) {
    const T k3y3 = p[2] * u[2], k3y2 = p[2] * u[1], k2y2x2 = T(2) * p[1] * u[1];
    o[0] = p[0] * (w[1] - w[0]);
    o[1] = M<T>::fma(k3y3, w[0] - w[1], k2y2x2 * (w[2] - w[1]));
    o[2] = k3y2 * (w[0] - w[1]);
  }
  static __device__ __forceinline__ void vjp_p(const T* u, const T*, T, const T* w, T* o) {
    o[0] = u[0] * (w[1] - w[0]);
    o[1] = u[1] * u[1] * (w[2] - w[1]);
    o[2] = u[1] * u[2] * (w[0] - w[1]);
  }
};

template <class T>
struct GBM {
  static constexpr int D = 1, P = 2, NW = 1;
  static constexpr bool autonomous = true, has_noise = true, sde_only = false, has_event = false;
  static constexpr bool stiff_only = false;
  static __device__ __forceinline__ void f(const T* u, const T* p, T, T* du) { du[0] = p[0] * u[0]; }
  // a = mu X, b = (sigma X) sqrt(h) Z
  static __device__ __forceinline__ void sde(const T* u, const T* p, T, T sq, const T* z, T* a,
                                             T* b) {
    a[0] = p[0] * u[0];
    b[0] = ((p[1] * u[0]) * sq) * z[0];
  }
  // diagonal noise: component j's diffusion b_j (the weak order 2 step evaluates it at shifted
  // states)
  static __device__ __forceinline__ void diag_b(const T* u, const T* p, T, T* b) {
    b[0] = p[1] * u[0];
  }
  static __device__ __forceinline__ void jac(const T*, const T* p, T, T* J) { J[0] = p[0]; }
  static __device__ __forceinline__ void vjp_u(const T*, const T* p, T, const T* w, T* o) {
    o[0] = p[0] * w[0];
  }
  static __device__ __forceinline__ void vjp_p(const T* u, const T*, T, const T* w, T* o) {
    o[0] = u[0] * w[0];
    o[1] = T(0);
  }
};

// Sigma-factor stress-response CRN (Appendix, SDE models) in the Chemical Langevin form:
// u = ([sigma], A1, A2, A3), p = (S, D, tau, nu0, n, eta), 8 Wiener processes.
//   a = (nu0 + H - [sigma], ([sigma] - A1)/tau, (A1 - A2)/tau, (A2 - A3)/tau),
//   H = (S[sigma])^n / ((S[sigma])^n + (D A3)^n + 1);
//   b_sigma = eta sq (sqrt(nu0 + H) z1 - sqrt([sigma]) z2),
//   b_Ai    = eta sq (sqrt(A_{i-1}/tau) z_{2i+1} - sqrt(A_i/tau) z_{2i+2}),  A_0 = [sigma].
// Square-root arguments and Hill bases are clamped at 0 (the form is undefined for negative
// amounts, which a discrete path can reach).  sqrt(x/tau) is formed as sqrt(x) sqrt(1/tau),
// so each amount's square root serves both terms it appears in.
// In float the powers are ex2(n lg2 x), the division and the square roots the MUFU forms:
// relative error <= ~5e-6 in (S[sigma])^n for the table's ranges (n lg2 x <= ~30, lg2 and
// ex2 good to 2^-22), ~1 ulp elsewhere -- far below the step's own O(h) error and inside the
// FP32 parity bounds.  Double keeps the correctly rounded library functions.
template <class T>
struct CRN {
  static constexpr int D = 4, P = 6, NW = 8;
  static constexpr bool autonomous = true, has_noise = true, sde_only = true, has_event = false;
  static constexpr bool stiff_only = false;
  static __device__ __forceinline__ T hill(const T* u, const T* p) {
    const T x = M<T>::fast_pow(M<T>::max(p[0] * u[0], T(0)), p[4]);
    const T y = M<T>::fast_pow(M<T>::max(p[1] * u[3], T(0)), p[4]);
    return M<T>::fast_div(x, (x + y) + T(1));
  }
  static __device__ __forceinline__ void drift(const T* u, const T* p, T H, T* a) {
    const T rt = M<T>::rcp(p[2]);
    a[0] = (p[3] + H) - u[0];
    a[1] = (u[0] - u[1]) * rt;
    a[2] = (u[1] - u[2]) * rt;
    a[3] = (u[2] - u[3]) * rt;
  }
  static __device__ __forceinline__ void f(const T* u, const T* p, T, T* du) {
    drift(u, p, hill(u, p), du);
  }
  static __device__ __forceinline__ T sqrt0(T x) { return M<T>::fast_sqrt(M<T>::max(x, T(0))); }
  static __device__ __forceinline__ void sde(const T* u, const T* p, T, T sq, const T* z, T* a,
                                             T* b) {
    const T H = hill(u, p);
    drift(u, p, H, a);
    const T e = p[5] * sq;
    const T er = e * M<T>::sqrt(M<T>::rcp(p[2]));  // eta sq / sqrt(tau)
    const T r0 = sqrt0(p[3] + H), r1 = sqrt0(u[0]), r2 = sqrt0(u[1]), r3 = sqrt0(u[2]),
            r4 = sqrt0(u[3]);
    b[0] = e * M<T>::fma(r0, z[0], -(r1 * z[1]));
    b[1] = er * M<T>::fma(r1, z[2], -(r2 * z[3]));
    b[2] = er * M<T>::fma(r2, z[4], -(r3 * z[5]));
    b[3] = er * M<T>::fma(r3, z[6], -(r4 * z[7]));
  }
};

// Bouncing ball (Sec. 6.5 event handling; Appendix, bouncing-ball problem): u = (x, v),
// p = (g, e); dx/dt = v, dv/dt = -g.  Event: the condition x = 0 reached from above
// triggers the affect v <- -e v (e the coefficient of restitution).  Adaptive Tsit5 only:
// the event is located on the step's dense output.
template <class T>
struct Ball {
  static constexpr int D = 2, P = 2, NW = 0;
  static constexpr bool autonomous = true, has_noise = false, sde_only = false, has_event = true;
  static constexpr bool stiff_only = false;
  static __device__ __forceinline__ void f(const T* u, const T* p, T, T* du) {
    du[0] = u[1];
    du[1] = -p[0];
  }
  static __device__ __forceinline__ T event_condition(const T* u, const T*, T) { return u[0]; }
  static __device__ __forceinline__ void event_affect(T* u, const T* p, T) { u[1] = -p[1] * u[1]; }
};

// The paper's stiff test models (Appendix): Oregonator (D = 3), HIRES (D = 8), POLLU
// (D = 20).  f and the Jacobian df/du (row-major); Rosenbrock23 and the explicit methods
// integrate them.
template <class T>
struct Orego {  // p = (k1, k2, k3); the first equation's sign read as + (Field-Noyes)
  static constexpr int D = 3, P = 3, NW = 0;
  static constexpr bool autonomous = true, has_noise = false, sde_only = false, has_event = false;
  static constexpr bool stiff_only = false;
  static __device__ __forceinline__ void f(const T* y, const T* k, T, T* dy) {
    dy[0] = k[0] * (y[1] + y[0] * (T(1) - k[1] * y[0] - y[1]));
    dy[1] = (y[2] - (T(1) + y[0]) * y[1]) / k[0];
    dy[2] = k[2] * (y[0] - y[2]);
  }
  static __device__ __forceinline__ void jac(const T* y, const T* k, T, T* J) {
    J[0] = k[0] * (T(1) - T(2) * k[1] * y[0] - y[1]);
    J[1] = k[0] * (T(1) - y[0]);
    J[2] = T(0);
    J[3] = -y[1] / k[0];
    J[4] = -(T(1) + y[0]) / k[0];
    J[5] = T(1) / k[0];
    J[6] = k[2];
    J[7] = T(0);
    J[8] = -k[2];
  }
};

template <class T>
struct Hires {  // p = the 12 distinct rate constants c1..c12 in order of appearance
  static constexpr int D = 8, P = 12, NW = 0;
  static constexpr bool autonomous = true, has_noise = false, sde_only = false, has_event = false;
  static constexpr bool stiff_only = true;  // Rosenbrock methods only, one per thread
  static __device__ __forceinline__ void f(const T* y, const T* c, T, T* dy) {
    const T r = c[9] * y[5] * y[7];
    dy[0] = -c[0] * y[0] + c[1] * y[1] + c[2] * y[2] + c[3];
    dy[1] = c[0] * y[0] - c[4] * y[1];
    dy[2] = -c[5] * y[2] + c[1] * y[3] + c[6] * y[4];
    dy[3] = c[2] * y[1] + c[0] * y[2] - c[7] * y[3];
    dy[4] = -c[8] * y[4] + c[1] * y[5] + c[1] * y[6];
    dy[5] = -r + c[10] * y[3] + c[0] * y[4] - c[1] * y[5] + c[10] * y[6];
    dy[6] = r - c[11] * y[6];
    dy[7] = -r + c[11] * y[6];
  }
  // The Jacobian's entries as add(row, col, 1, value) with compile-time row and col (each
  // entry once, so J[r][c] = fma(1, value, 0) = value).
  template <class ADD>
  static __device__ __forceinline__ void jac_visit(const T* y, const T* c, T, ADD&& add) {
    const T one(1);
    auto e = [&](auto r, auto col, T v) { add(r, col, one, v); };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    using I4 = std::integral_constant<int, 4>;
    using I5 = std::integral_constant<int, 5>;
    using I6 = std::integral_constant<int, 6>;
    using I7 = std::integral_constant<int, 7>;
    e(I0(), I0(), -c[0]); e(I0(), I1(), c[1]); e(I0(), I2(), c[2]);
    e(I1(), I0(), c[0]); e(I1(), I1(), -c[4]);
    e(I2(), I2(), -c[5]); e(I2(), I3(), c[1]); e(I2(), I4(), c[6]);
    e(I3(), I1(), c[2]); e(I3(), I2(), c[0]); e(I3(), I3(), -c[7]);
    e(I4(), I4(), -c[8]); e(I4(), I5(), c[1]); e(I4(), I6(), c[1]);
    e(I5(), I3(), c[10]); e(I5(), I4(), c[0]); e(I5(), I5(), -c[9] * y[7] - c[1]);
    e(I5(), I6(), c[10]); e(I5(), I7(), -c[9] * y[5]);
    e(I6(), I5(), c[9] * y[7]); e(I6(), I6(), -c[11]); e(I6(), I7(), c[9] * y[5]);
    e(I7(), I5(), -c[9] * y[7]); e(I7(), I6(), c[11]); e(I7(), I7(), -c[9] * y[5]);
  }
  static __host__ __device__ constexpr Pattern<8> jac_pattern() {
    Pattern<8> s{};
    constexpr int nz[25][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 0}, {1, 1}, {2, 2}, {2, 3},
                               {2, 4}, {3, 1}, {3, 2}, {3, 3}, {4, 4}, {4, 5}, {4, 6},
                               {5, 3}, {5, 4}, {5, 5}, {5, 6}, {5, 7}, {6, 5}, {6, 6},
                               {6, 7}, {7, 5}, {7, 6}, {7, 7}};
    for (int i = 0; i < 25; ++i) s.nz[nz[i][0]][nz[i][1]] = true;
    return s;
  }
  static __device__ __forceinline__ void jac(const T* y, const T* c, T t, T* J) {
#pragma unroll
    for (int i = 0; i < 64; ++i) J[i] = T(0);
    jac_visit(y, c, t, [&](auto r, auto col, T nu, T v) {
      J[decltype(r)::value * 8 + decltype(col)::value] =
          M<T>::fma(nu, v, J[decltype(r)::value * 8 + decltype(col)::value]);
    });
  }
};

// POLLU as its 25 mass-action reactions: rate r_j = k_j y_a (y_b), and the change of each
// species per unit of r_j (the printed equations are exactly the sum over the reactions).
struct PolluRx {
  int a, b, n;  // reactants (b = -1: first order), number of species changed
  int sp[5];
  int nu[5];
};
__host__ __device__ constexpr PolluRx pollu_rx(int j) {
  constexpr PolluRx R[25] = {
      {0, -1, 3, {0, 1, 2}, {-1, 1, 1}},          {1, 3, 3, {0, 1, 3}, {1, -1, -1}},
      {4, 1, 4, {0, 1, 4, 5}, {1, -1, -1, 1}},    {6, -1, 3, {4, 6, 7}, {2, -1, 1}},
      {6, -1, 2, {6, 7}, {-1, 1}},                {6, 5, 4, {4, 5, 6, 7}, {1, -1, -1, 1}},
      {8, -1, 4, {4, 7, 8, 9}, {1, 1, -1, 1}},    {8, 5, 3, {5, 8, 10}, {-1, -1, 1}},
      {10, 1, 5, {0, 1, 9, 10, 11}, {1, -1, 1, -1, 1}},
      {10, 0, 3, {0, 10, 12}, {-1, -1, 1}},       {12, -1, 3, {0, 10, 12}, {1, 1, -1}},
      {9, 1, 4, {0, 1, 9, 13}, {1, -1, -1, 1}},   {13, -1, 3, {4, 6, 13}, {1, 1, -1}},
      {0, 5, 3, {0, 5, 14}, {-1, -1, 1}},         {2, -1, 2, {2, 3}, {-1, 1}},
      {3, -1, 2, {3, 15}, {-1, 1}},               {3, -1, 2, {2, 3}, {1, -1}},
      {15, -1, 2, {5, 15}, {2, -1}},              {15, -1, 2, {2, 15}, {1, -1}},
      {16, 5, 4, {4, 5, 16, 17}, {1, -1, -1, 1}}, {18, -1, 2, {1, 18}, {1, -1}},
      {18, -1, 3, {0, 2, 18}, {1, 1, -1}},        {0, 3, 3, {0, 3, 18}, {-1, -1, 1}},
      {18, 0, 3, {0, 18, 19}, {-1, -1, 1}},       {19, -1, 3, {0, 18, 19}, {1, 1, -1}}};
  return R[j];
}

template <class T>
struct Pollu {  // p = (k1..k25)
  static constexpr int D = 20, P = 25, NW = 0;
  static constexpr bool autonomous = true, has_noise = false, sde_only = false, has_event = false;
  static constexpr bool stiff_only = true;  // Rosenbrock methods only, one per thread
  static __device__ __forceinline__ void f(const T* y, const T* k, T, T* dy) {
#pragma unroll
    for (int i = 0; i < 20; ++i) dy[i] = T(0);
#pragma unroll
    for (int j = 0; j < 25; ++j) {
      const PolluRx r = pollu_rx(j);
      const T rate = r.b < 0 ? k[j] * y[r.a] : k[j] * y[r.a] * y[r.b];
#pragma unroll
      for (int m = 0; m < 5; ++m)
        if (m < r.n) dy[r.sp[m]] = M<T>::fma(T(r.nu[m]), rate, dy[r.sp[m]]);
    }
  }
  // The Jacobian as a sum over the reactions: reaction j adds nu_m d(r_j)/d(y_a) (and
  // d(r_j)/d(y_b)) to row sp_m, as add(row, col, nu, derivative) with compile-time row and
  // col, in reaction order.
  template <class ADD>
  static __device__ __forceinline__ void jac_visit(const T* y, const T* k, T, ADD&& add) {
    static_for<0, 25>([&](auto J) {
      constexpr int j = decltype(J)::value;
      constexpr PolluRx r = pollu_rx(j);
      const T dra = r.b < 0 ? k[j] : k[j] * y[r.b < 0 ? 0 : r.b];
      const T drb = r.b < 0 ? T(0) : k[j] * y[r.a];
      static_for<0, r.n>([&](auto Q) {
        constexpr PolluRx x = pollu_rx(j);  // (a lambda cannot read the enclosing one's r at
                                            // compile time)
        constexpr int q = decltype(Q)::value;
        constexpr int row = x.sp[q];
        add(std::integral_constant<int, row>(), std::integral_constant<int, x.a>(), T(x.nu[q]),
            dra);
        if constexpr (x.b >= 0)
          add(std::integral_constant<int, row>(), std::integral_constant<int, (x.b < 0 ? 0 : x.b)>(),
              T(x.nu[q]), drb);
      });
    });
  }
  static __host__ __device__ constexpr Pattern<20> jac_pattern() {
    Pattern<20> s{};
    for (int j = 0; j < 25; ++j) {
      const PolluRx r = pollu_rx(j);
      for (int m = 0; m < r.n; ++m) {
        s.nz[r.sp[m]][r.a] = true;
        if (r.b >= 0) s.nz[r.sp[m]][r.b] = true;
      }
    }
    return s;
  }
  static __device__ __forceinline__ void jac(const T* y, const T* k, T t, T* J) {
#pragma unroll
    for (int i = 0; i < 400; ++i) J[i] = T(0);
    jac_visit(y, k, t, [&](auto r, auto c, T nu, T v) {
      J[decltype(r)::value * 20 + decltype(c)::value] =
          M<T>::fma(nu, v, J[decltype(r)::value * 20 + decltype(c)::value]);
    });
  }
};

// ------------------------------------------------------------------------------------------
// Tsitouras 5(4) coefficients (Tsitouras 2011; GPUTsit5, Sec. 5.2.1).  BT_i = bhat_i - b_i.
struct Ts5 {
  static constexpr double c2 = 0.161, c3 = 0.327, c4 = 0.9, c5 = 0.9800255409045097;
  static constexpr double a21 = 0.161;
  static constexpr double a31 = -0.008480655492356989, a32 = 0.335480655492357;
  static constexpr double a41 = 2.897153057105493, a42 = -6.359448489975075,
                          a43 = 4.3622954328695815;
  static constexpr double a51 = 5.325864828439257, a52 = -11.748883564062828,
                          a53 = 7.4955393428898365, a54 = -0.09249506636175525;
  static constexpr double a61 = 5.86145544294642, a62 = -12.92096931784711,
                          a63 = 8.159367898576159, a64 = -0.071584973281401,
                          a65 = -0.028269050394068383;
  static constexpr double a71 = 0.09646076681806523, a72 = 0.01, a73 = 0.4798896504144996,
                          a74 = 1.379008574103742, a75 = -3.290069515436081,
                          a76 = 2.324710524099774;
  static constexpr double bt1 = 0.09468075576583945 - a71, bt2 = 0.009183565540343254 - a72,
                          bt3 = 0.4877705284247616 - a73, bt4 = 1.234297566930479 - a74,
                          bt5 = -2.7077123499835256 - a75, bt6 = 1.866628418170587 - a76,
                          bt7 = 0.015151515151515152;
};

// One Tsit5 step: U_i = u + h sum_j a_ij k_j, k_i = f(U_i, t + c_i h) (Sec. 3.1); stage 7 is
// u_{n+1} itself (FSAL) and k7 = f(u_{n+1}).  With WANT_ERR, es = sum_j (bhat_j - b_j) k_j
// (the error estimate is h * es).
template <class RHS, class T, bool WANT_ERR>
__device__ __forceinline__ void tsit5_step(const T* u, const T* p, T t, T h, const T* k1,
                                           T* unew, T* es, T* k7, T* kmid = nullptr) {
  constexpr int D = RHS::D;
  typedef M<T> m;
  T U[D], k2[D], k3[D], k4[D], k5[D], k6[D];
#pragma unroll
  for (int j = 0; j < D; ++j) U[j] = m::fma(h, T(Ts5::a21) * k1[j], u[j]);
  RHS::f(U, p, t + T(Ts5::c2) * h, k2);
#pragma unroll
  for (int j = 0; j < D; ++j)
    U[j] = m::fma(h, m::fma(T(Ts5::a32), k2[j], T(Ts5::a31) * k1[j]), u[j]);
  RHS::f(U, p, t + T(Ts5::c3) * h, k3);
#pragma unroll
  for (int j = 0; j < D; ++j)
    U[j] = m::fma(h, m::fma(T(Ts5::a43), k3[j], m::fma(T(Ts5::a42), k2[j], T(Ts5::a41) * k1[j])),
                  u[j]);
  RHS::f(U, p, t + T(Ts5::c4) * h, k4);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    T s = T(Ts5::a51) * k1[j];
    s = m::fma(T(Ts5::a52), k2[j], s);
    s = m::fma(T(Ts5::a53), k3[j], s);
    s = m::fma(T(Ts5::a54), k4[j], s);
    U[j] = m::fma(h, s, u[j]);
  }
  RHS::f(U, p, t + T(Ts5::c5) * h, k5);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    T s = T(Ts5::a61) * k1[j];
    s = m::fma(T(Ts5::a62), k2[j], s);
    s = m::fma(T(Ts5::a63), k3[j], s);
    s = m::fma(T(Ts5::a64), k4[j], s);
    s = m::fma(T(Ts5::a65), k5[j], s);
    U[j] = m::fma(h, s, u[j]);
  }
  RHS::f(U, p, t + h, k6);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    T s = T(Ts5::a71) * k1[j];
    s = m::fma(T(Ts5::a72), k2[j], s);
    s = m::fma(T(Ts5::a73), k3[j], s);
    s = m::fma(T(Ts5::a74), k4[j], s);
    s = m::fma(T(Ts5::a75), k5[j], s);
    s = m::fma(T(Ts5::a76), k6[j], s);
    unew[j] = m::fma(h, s, u[j]);
  }
  RHS::f(unew, p, t + h, k7);
  if (kmid) {  // stages 2..6 for the dense output
#pragma unroll
    for (int j = 0; j < D; ++j) {
      kmid[j] = k2[j];
      kmid[D + j] = k3[j];
      kmid[2 * D + j] = k4[j];
      kmid[3 * D + j] = k5[j];
      kmid[4 * D + j] = k6[j];
    }
  }
  if (WANT_ERR) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      T s = T(Ts5::bt1) * k1[j];
      s = m::fma(T(Ts5::bt2), k2[j], s);
      s = m::fma(T(Ts5::bt3), k3[j], s);
      s = m::fma(T(Ts5::bt4), k4[j], s);
      s = m::fma(T(Ts5::bt5), k5[j], s);
      s = m::fma(T(Ts5::bt6), k6[j], s);
      s = m::fma(T(Ts5::bt7), k7[j], s);
      es[j] = s;
    }
  }
}

// Dense output of a Tsit5 step (Sec. 5.1.1 solution storage; the pair's interpolant is not
// printed in the paper): u(t_n + theta h) = u_n + h sum_i b_i(theta) k_i with
// b_i(theta) = theta (r_i1 + theta (r_i2 + theta (r_i3 + theta r_i4))).  The r are the C1
// continuous extension of order 4: for every theta the elementary-weight conditions of the
// 8 rooted trees of order <= 4 hold, b_i(1) = b_i, b_i'(0) = [i = 1], b_i'(1) = [i = 7]; of
// the one-parameter family these leave, the member with the smallest integrated squared
// 5th-order defect (derived in 40-digit arithmetic from the pair's coefficients).
__host__ __device__ constexpr double ts5_dense(int i, int q) {
  constexpr double r[7][4] = {
      {1.0, -2.7697190760997743, 2.925281219471809, -1.0591013765539699},
      {0.0, 0.12894208371183252, -0.2178841674236653, 0.09894208371183272},
      {0.0, 3.956917849412212, -5.994277097166426, 2.5172488981687136},
      {0.0, -12.899911070336683, 31.315856437088335, -17.03693679264791},
      {0.0, 39.47651640903875, -92.11331087982184, 49.346724955347},
      {0.0, -29.443928026595056, 68.1866981495892, -36.418059598894374},
      {0.0, 1.5511818308687129, -4.102363661737424, 2.551181830868712}};
  return r[i][q];
}

// The same interpolant as a polynomial in theta, u(theta) = u_n + sum_{q=1..4} theta^q c_q
// with c_q = h sum_i r_iq k_i (dense_coeffs once per step, dense_poly per point): the form
// dense saving and event location evaluate.
//
// Events (Sec. 6.5): a condition g(u, p, t) crossing zero from above inside an accepted step
// triggers the model's affect.  The condition is
// checked at theta = j / kEventPoints (u_n and u_{n+1} themselves at the ends); the first
// interval with g > 0 at its left end and g <= 0 at its right end is narrowed by the Illinois
// method (regula falsi that halves the value kept at an end surviving two iterations in a
// row; Dowell & Jarratt 1971) until it is at most 4 eps wide or after 100 iterations.  The
// event sits at the interval's right end.
constexpr int kEventPoints = 10;

template <class RHS, class T>
__device__ __forceinline__ void dense_coeffs(T h, const T* k1, const T* kmid, const T* k7,
                                             T (*c)[RHS::D]) {
  constexpr int D = RHS::D;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      T s = T(ts5_dense(0, q)) * k1[j];
#pragma unroll
      for (int i = 1; i < 6; ++i) s = M<T>::fma(T(ts5_dense(i, q)), kmid[(i - 1) * D + j], s);
      s = M<T>::fma(T(ts5_dense(6, q)), k7[j], s);
      c[q][j] = h * s;
    }
}

template <class RHS, class T>
__device__ __forceinline__ void dense_poly(const T* u, const T (*c)[RHS::D], T th, T* out) {
#pragma unroll
  for (int j = 0; j < RHS::D; ++j)
    out[j] = M<T>::fma(th, M<T>::fma(th, M<T>::fma(th, M<T>::fma(th, c[3][j], c[2][j]), c[1][j]),
                                     c[0][j]),
                       u[j]);
}

// theta in (0, 1] of the first crossing from above in the step, or -1 for none
template <class RHS, class T>
__device__ T find_event(const T* u, const T* unew, const T* p, T tn, T h,
                        const T (*c)[RHS::D]) {
  T w[RHS::D];
  T a = T(0), ga = RHS::event_condition(u, p, tn);
  for (int j = 1; j <= kEventPoints; ++j) {
    T b0, gb0;
    if (j == kEventPoints) {
      b0 = T(1);
      gb0 = RHS::event_condition(unew, p, tn + h);
    } else {
      b0 = T(j) / T(kEventPoints);
      dense_poly<RHS, T>(u, c, b0, w);
      gb0 = RHS::event_condition(w, p, tn + b0 * h);
    }
    if (ga > T(0) && gb0 <= T(0)) {
      T b = b0, gb = gb0;
      int side = 0;
      const T width = T(4) * (sizeof(T) == 4 ? T(1.1920928955078125e-07) : T(2.220446049250313e-16));
      for (int it = 0; it < 100 && b - a > width; ++it) {
        T x = (a * gb - b * ga) / (gb - ga);
        if (!(x > a && x < b)) x = (a + b) * T(0.5);
        dense_poly<RHS, T>(u, c, x, w);
        const T gx = RHS::event_condition(w, p, tn + x * h);
        if (gx > T(0)) {
          a = x;
          ga = gx;
          if (side == 1) gb *= T(0.5);
          side = 1;
        } else {
          b = x;
          gb = gx;
          if (side == -1) ga *= T(0.5);
          side = -1;
        }
      }
      return b;
    }
    a = b0;
    ga = gb0;
  }
  return T(-1);
}

// Classic RK4 step.
template <class RHS, class T>
__device__ __forceinline__ void rk4_step(const T* u, const T* p, T t, T h, T* unew) {
  constexpr int D = RHS::D;
  typedef M<T> m;
  T k1[D], k2[D], k3[D], k4[D], U[D];
  const T hh = T(0.5) * h;
  RHS::f(u, p, t, k1);
#pragma unroll
  for (int j = 0; j < D; ++j) U[j] = m::fma(hh, k1[j], u[j]);
  RHS::f(U, p, t + hh, k2);
#pragma unroll
  for (int j = 0; j < D; ++j) U[j] = m::fma(hh, k2[j], u[j]);
  RHS::f(U, p, t + hh, k3);
#pragma unroll
  for (int j = 0; j < D; ++j) U[j] = m::fma(h, k3[j], u[j]);
  RHS::f(U, p, t + h, k4);
  const T h6 = h * T(1.0 / 6.0);
#pragma unroll
  for (int j = 0; j < D; ++j) unew[j] = m::fma(h6, (k1[j] + k4[j]) + T(2) * (k2[j] + k3[j]), u[j]);
}

// ------------------------------------------------------------------------------------------
// Dense LU with partial pivoting, small D, fully unrolled; the row exchanges are done with
// selects so that no lane branches.  Ties keep the lower row (strict > comparison).
template <class T, int D>
struct LU {
  T a[D][D];          // L (unit, strictly lower) and U (upper; diagonal stored as reciprocal)
  bool sw[D][D];      // sw[c][r]: rows c and r were exchanged for column c (at most one r)

  __device__ __forceinline__ void factor(T (&W)[D][D]) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      // pivot: the first row of largest |W[r][c]|, r >= c; then exchange it with row c
      T big = M<T>::abs(W[c][c]);
      int best = c;
#pragma unroll
      for (int r = c + 1; r < D; ++r) {
        const T v = M<T>::abs(W[r][c]);
        const bool g = v > big;
        big = g ? v : big;
        best = g ? r : best;
      }
#pragma unroll
      for (int r = c + 1; r < D; ++r) {
        const bool x = (best == r);
        sw[c][r] = x;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const T wc = W[c][j], wr = W[r][j];
          W[c][j] = x ? wr : wc;
          W[r][j] = x ? wc : wr;
        }
      }
      const T inv = M<T>::rcp(W[c][c]);
      W[c][c] = inv;
#pragma unroll
      for (int r = c + 1; r < D; ++r) {
        const T l = W[r][c] * inv;
        W[r][c] = l;
#pragma unroll
        for (int j = c + 1; j < D; ++j) W[r][j] = M<T>::fma(-l, W[c][j], W[r][j]);
      }
    }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int j = 0; j < D; ++j) a[r][j] = W[r][j];
  }

  // x = W^{-1} b
  __device__ __forceinline__ void solve(const T* b, T* x) const {
    T y[D];
#pragma unroll
    for (int r = 0; r < D; ++r) y[r] = b[r];
    // apply the row exchanges in elimination order, then forward substitution with unit L
#pragma unroll
    for (int c = 0; c < D; ++c) {
#pragma unroll
      for (int r = c + 1; r < D; ++r) {
        const T yc = y[c], yr = y[r];
        y[c] = sw[c][r] ? yr : yc;
        y[r] = sw[c][r] ? yc : yr;
      }
    }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int j = 0; j < r; ++j) y[r] = M<T>::fma(-a[r][j], y[j], y[r]);
#pragma unroll
    for (int r = D - 1; r >= 0; --r) {
      T v = y[r];
#pragma unroll
      for (int j = r + 1; j < D; ++j) v = M<T>::fma(-a[r][j], x[j], v);
      x[r] = v * a[r][r];
    }
  }
};

// The same factorisation and solve for larger D (8 and up) as loops over a local-memory
// matrix: the fully unrolled, select-based form above would need D^2 registers and D^3 / 2
// selects (at D = 20 it spills and takes minutes to compile).  Same pivot rule, same operation
// order, so the same results.
template <class T, int D>
struct LUDyn {
  T a[D][D];
  int piv[D];  // row exchanged with row c for column c (c itself: none)

  // factor a (filled by the caller) in place
  __device__ void factor() {
#pragma unroll 1
    for (int c = 0; c < D; ++c) {
      T big = M<T>::abs(a[c][c]);
      int best = c;
#pragma unroll 1
      for (int r = c + 1; r < D; ++r) {
        const T v = M<T>::abs(a[r][c]);
        if (v > big) {
          big = v;
          best = r;
        }
      }
      piv[c] = best;
      if (best != c) {
#pragma unroll 4
        for (int j = 0; j < D; ++j) {
          const T t = a[c][j];
          a[c][j] = a[best][j];
          a[best][j] = t;
        }
      }
      const T inv = M<T>::rcp(a[c][c]);
      a[c][c] = inv;
#pragma unroll 1
      for (int r = c + 1; r < D; ++r) {
        // a zero below the pivot leaves its row as it is (fma(-0, x, y) = y for finite x):
        // the stiff models' matrices are mostly zeros, in the same places for every
        // trajectory, so the skip is the same across the warp
        if (a[r][c] == T(0)) continue;
        const T l = a[r][c] * inv;
        a[r][c] = l;
        // independent across j: unrolled so several local-memory loads are in flight
#pragma unroll 4
        for (int j = c + 1; j < D; ++j) a[r][j] = M<T>::fma(-l, a[c][j], a[r][j]);
      }
    }
  }

  __device__ void solve(const T* b, T* x) const {
    T y[D];
#pragma unroll
    for (int r = 0; r < D; ++r) y[r] = b[r];
#pragma unroll 1
    for (int c = 0; c < D; ++c) {
      const int q = piv[c];
      if (q != c) {
        const T t = y[c];
        y[c] = y[q];
        y[q] = t;
      }
    }
#pragma unroll 1
    for (int r = 0; r < D; ++r)
#pragma unroll 4
      for (int j = 0; j < r; ++j) y[r] = M<T>::fma(-a[r][j], y[j], y[r]);
#pragma unroll 1
    for (int r = D - 1; r >= 0; --r) {
      T v = y[r];
#pragma unroll 4
      for (int j = r + 1; j < D; ++j) v = M<T>::fma(-a[r][j], x[j], v);
      x[r] = v * a[r][r];
    }
  }
};

// ------------------------------------------------------------------------------------------
// Sparse LU of W = I - hg J on a model's fixed Jacobian pattern (the large stiff models,
// Appendix: HIRES, POLLU).  Everything about the structure is decided at compile time:
//  * the elimination order: greedy minimum degree on the symmetrised pattern (the variable
//    with the fewest remaining neighbours first, ties to the lower index; its neighbours then
//    form a clique);
//  * the filled pattern of the symmetrically permuted matrix P W P^T (symbolic elimination)
//    and a compressed slot for each of its entries;
//  * the factorisation and the two triangular solves as flat operation lists, expanded into
//    straight-line code with constant slots (no index arithmetic, no zero tests).
// The numeric factorisation exchanges no rows and checks, column by column, that partial
// pivoting would not exchange any either (|a_kk| >= |a_rk| for every r below k; a NaN fails):
// when every check passes the factors are those of partial pivoting on P W P^T.  When one
// fails the step factors W again, densely and with row exchanges (LUDyn).  On POLLU in
// natural order partial pivoting exchanges rows in most factorisations and the factors fill
// 262 of 400 entries; in the minimum-degree order the factors hold 109 entries, the
// elimination takes 162 multiply-adds, and the checks held on every factorisation of the
// oracle's solves (Rosenbrock23, Rodas4, Rodas5P at tolerance 1e-6, also at 3x the step).

enum SpKind : short { SP_CHECK, SP_RCP, SP_MUL, SP_FMA, SP_DIAG };

struct SpOp {
  short kind, d, s1, s2;
};

template <int D>
struct SpPlan {
  static constexpr int MAXOP = 1024;
  int order[D];      // order[k]: the variable eliminated k-th
  int pos[D];        // pos[v]: the position of variable v
  int slot[D][D];    // compressed slot of entry (position r, position c); -1 outside the fill
  int nnz;
  bool w_entry[D * D];  // slot holds a structural entry of W (of J, or the diagonal)
  bool is_diag[D * D];
  SpOp fac[MAXOP];   // factorisation: checks, reciprocal pivots, multipliers, updates
  int nfac;
  SpOp fwd[D * D];   // forward substitution with unit L (positions)
  int nfwd;
  SpOp bwd[D * D];   // back substitution with U (diagonal stored inverted)
  int nbwd;
};

template <int D>
__host__ __device__ constexpr SpPlan<D> make_sp_plan(const Pattern<D> J) {
  SpPlan<D> P{};
  // minimum degree on the symmetrised pattern
  bool G[D][D] = {};
  bool alive[D] = {};
  for (int r = 0; r < D; ++r) {
    alive[r] = true;
    for (int c = 0; c < D; ++c) G[r][c] = J.nz[r][c] || J.nz[c][r] || r == c;
  }
  for (int k = 0; k < D; ++k) {
    int best = -1, bdeg = D + 1;
    for (int v = 0; v < D; ++v) {
      if (!alive[v]) continue;
      int deg = 0;
      for (int u = 0; u < D; ++u) deg += (alive[u] && G[v][u]) ? 1 : 0;
      if (deg < bdeg) {
        bdeg = deg;
        best = v;
      }
    }
    P.order[k] = best;
    P.pos[best] = k;
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b)
        if (alive[a] && alive[b] && a != best && b != best && G[best][a] && G[best][b])
          G[a][b] = true;
    alive[best] = false;
  }
  // filled pattern of P W P^T
  bool F[D][D] = {};
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) F[r][c] = J.nz[P.order[r]][P.order[c]] || r == c;
  bool W[D][D] = {};
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) W[r][c] = F[r][c];
  for (int k = 0; k < D; ++k)
    for (int r = k + 1; r < D; ++r)
      if (F[r][k])
        for (int j = k + 1; j < D; ++j)
          if (F[k][j]) F[r][j] = true;
  int e = 0;
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      P.slot[r][c] = F[r][c] ? e : -1;
      if (F[r][c]) {
        P.w_entry[e] = W[r][c];
        P.is_diag[e] = r == c;
        ++e;
      }
    }
  P.nnz = e;
  // factorisation, right-looking in position order
  int n = 0;
  for (int k = 0; k < D; ++k) {
    const short kk = (short)P.slot[k][k];
    for (int r = k + 1; r < D; ++r)
      if (F[r][k]) P.fac[n++] = SpOp{SP_CHECK, kk, (short)P.slot[r][k], 0};
    P.fac[n++] = SpOp{SP_RCP, kk, 0, 0};
    for (int r = k + 1; r < D; ++r) {
      if (!F[r][k]) continue;
      const short rk = (short)P.slot[r][k];
      P.fac[n++] = SpOp{SP_MUL, rk, kk, 0};
      for (int j = k + 1; j < D; ++j)
        if (F[k][j]) P.fac[n++] = SpOp{SP_FMA, (short)P.slot[r][j], rk, (short)P.slot[k][j]};
    }
  }
  P.nfac = n;
  // solves, column-oriented (each finished unknown updates the rows that use it)
  n = 0;
  for (int k = 0; k < D; ++k)
    for (int r = k + 1; r < D; ++r)
      if (F[r][k]) P.fwd[n++] = SpOp{SP_FMA, (short)r, (short)P.slot[r][k], (short)k};
  P.nfwd = n;
  n = 0;
  for (int k = D - 1; k >= 0; --k) {
    P.bwd[n++] = SpOp{SP_DIAG, (short)k, (short)P.slot[k][k], 0};
    for (int r = 0; r < k; ++r)
      if (F[r][k]) P.bwd[n++] = SpOp{SP_FMA, (short)r, (short)P.slot[r][k], (short)k};
  }
  P.nbwd = n;
  return P;
}

template <class RHS>
struct SpPlanOf {
  static constexpr SpPlan<RHS::D> plan = make_sp_plan<RHS::D>(RHS::jac_pattern());
  static_assert(plan.nfac <= SpPlan<RHS::D>::MAXOP, "factorisation list too long");
};

template <class RHS>
struct HasSparseJac {
 private:
  template <class R>
  static constexpr bool test(decltype(R::jac_pattern())*) { return true; }
  template <class R>
  static constexpr bool test(...) { return false; }

 public:
  static constexpr bool value = test<RHS>(nullptr);
};

template <class RHS, class T>
struct SparseRosLU {
  static constexpr int D = RHS::D;
  typedef SpPlanOf<RHS> PL;
  T a[PL::plan.nnz];
  bool dense;       // a pivot check failed: lud holds the row-exchanging factorisation
  LUDyn<T, D> lud;

  // W = I - hg J at (u, p, t), factored
  __device__ __forceinline__ void factor(const T* u, const T* p, T t, T hg) {
    typedef M<T> m;
    static_for<0, PL::plan.nnz>([&](auto E) { a[decltype(E)::value] = T(0); });
    RHS::jac_visit(u, p, t, [&](auto R, auto C, T nu, T v) {
      constexpr int e = PL::plan.slot[PL::plan.pos[decltype(R)::value]][PL::plan.pos[decltype(C)::value]];
      static_assert(e >= 0, "a Jacobian entry outside the declared pattern");
      a[e] = m::fma(nu, v, a[e]);
    });
    static_for<0, PL::plan.nnz>([&](auto E) {
      constexpr int e = decltype(E)::value;
      constexpr bool diag = PL::plan.is_diag[e];
      if constexpr (PL::plan.w_entry[e]) a[e] = m::fma(-hg, a[e], diag ? T(1) : T(0));
    });
    bool bad = false;
    static_for<0, PL::plan.nfac>([&](auto I) {
      constexpr SpOp o = PL::plan.fac[decltype(I)::value];
      if constexpr (o.kind == SP_CHECK) {
        bad = bad || !(m::abs(a[o.s1]) <= m::abs(a[o.d]));
      } else if constexpr (o.kind == SP_RCP) {
        a[o.d] = m::rcp(a[o.d]);
      } else if constexpr (o.kind == SP_MUL) {
        a[o.d] = a[o.d] * a[o.s1];
      } else {
        a[o.d] = m::fma(-a[o.s1], a[o.s2], a[o.d]);
      }
    });
    dense = bad;
    if (bad) {  // partial pivoting would exchange rows here: the dense factorisation
      RHS::jac(u, p, t, &lud.a[0][0]);
#pragma unroll 1
      for (int r = 0; r < D; ++r)
#pragma unroll 1
        for (int c = 0; c < D; ++c) lud.a[r][c] = m::fma(-hg, lud.a[r][c], (r == c) ? T(1) : T(0));
      lud.factor();
    }
  }

  // x = W^{-1} b
  __device__ __forceinline__ void solve(const T* b, T* x) const {
    typedef M<T> m;
    if (dense) {
      lud.solve(b, x);
      return;
    }
    T y[D];
    static_for<0, D>([&](auto K) {
      constexpr int k = decltype(K)::value, v = PL::plan.order[k];
      y[k] = b[v];
    });
    static_for<0, PL::plan.nfwd>([&](auto I) {
      constexpr SpOp o = PL::plan.fwd[decltype(I)::value];
      y[o.d] = m::fma(-a[o.s1], y[o.s2], y[o.d]);
    });
    static_for<0, PL::plan.nbwd>([&](auto I) {
      constexpr SpOp o = PL::plan.bwd[decltype(I)::value];
      if constexpr (o.kind == SP_DIAG) {
        y[o.d] = y[o.d] * a[o.s1];
      } else {
        y[o.d] = m::fma(-a[o.s1], y[o.s2], y[o.d]);
      }
    });
    static_for<0, D>([&](auto K) {
      constexpr int k = decltype(K)::value, v = PL::plan.order[k];
      x[v] = y[k];
    });
  }
};

// W = I - hg J for a Rosenbrock step (hg = h times the method's diagonal coefficient), factored
// into lu: J and W in registers for small D, all in the one local-memory matrix for large D (a
// thread's footprint stays D^2 values, so the resident threads' matrices fit in L1).
template <class RHS, class T, class LUT>
__device__ __forceinline__ void ros_factor(const T* u, const T* p, T t, T hg, LUT& lu) {
  constexpr int D = RHS::D;
  typedef M<T> m;
  if constexpr (HasSparseJac<RHS>::value) {
    lu.factor(u, p, t, hg);
  } else if constexpr (D < 12) {
    T Jf[D * D];
    RHS::jac(u, p, t, Jf);
    T W[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) W[r][c] = m::fma(-hg, Jf[r * D + c], (r == c) ? T(1) : T(0));
    if constexpr (D < 8) {
      lu.factor(W);
    } else {
#pragma unroll
      for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) lu.a[r][c] = W[r][c];
      lu.factor();
    }
  } else {
    RHS::jac(u, p, t, &lu.a[0][0]);
#pragma unroll 1
    for (int r = 0; r < D; ++r)
#pragma unroll 1
      for (int c = 0; c < D; ++c) lu.a[r][c] = m::fma(-hg, lu.a[r][c], (r == c) ? T(1) : T(0));
    lu.factor();
  }
}

template <class T, int D>
using RosLU = typename std::conditional<(D < 8), LU<T, D>, LUDyn<T, D>>::type;

// the factorisation a Rosenbrock step of model RHS uses: the sparse one where the model
// declares its Jacobian pattern, else the dense one for its size
template <class RHS, class T>
using RosLUOf = typename std::conditional<HasSparseJac<RHS>::value, SparseRosLU<RHS, T>,
                                          RosLU<T, RHS::D>>::type;

// One Rosenbrock23 (ode23s) step from (u, t) with f0 = f(u, t); W = I - h d J:
//   k1 = W^-1 f0,  f1 = f(u + h/2 k1),  k2 = W^-1 (f1 - k1) + k1,  u_{n+1} = u + h k2,
//   f2 = f(u_{n+1}),  k3 = W^-1 (f2 - e32 (k2 - f1) - 2 (k1 - f0)),  err = h/6 (k1 - 2 k2 + k3).
// Autonomous models only (df/dt = 0).  Writes es = (k1 - 2 k2 + k3)/6 (err = h * es).
template <class RHS, class T>
__device__ __forceinline__ void ros23_step(const T* u, const T* p, T t, T h, const T* f0, T* unew,
                                           T* es, T* f2) {
  static_assert(RHS::autonomous, "Rosenbrock23 here assumes df/dt = 0");
  constexpr int D = RHS::D;
  typedef M<T> m;
  const T d = T(0.29289321881345247559915563789515);   // 1 / (2 + sqrt 2)
  const T e32 = T(7.4142135623730950488016887242097);  // 6 + sqrt 2
  const T hd = h * d;
  RosLUOf<RHS, T> lu;
  ros_factor<RHS, T>(u, p, t, hd, lu);
  T k1[D], k2[D], k3[D], f1[D], U[D], v[D];
  lu.solve(f0, k1);
  const T hh = T(0.5) * h;
#pragma unroll
  for (int j = 0; j < D; ++j) U[j] = m::fma(hh, k1[j], u[j]);
  RHS::f(U, p, t + hh, f1);
#pragma unroll
  for (int j = 0; j < D; ++j) v[j] = f1[j] - k1[j];
  lu.solve(v, k2);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    k2[j] += k1[j];
    unew[j] = m::fma(h, k2[j], u[j]);
  }
  RHS::f(unew, p, t + h, f2);
#pragma unroll
  for (int j = 0; j < D; ++j)
    v[j] = m::fma(-e32, k2[j] - f1[j], m::fma(T(-2), k1[j] - f0[j], f2[j]));
  lu.solve(v, k3);
#pragma unroll
  for (int j = 0; j < D; ++j) es[j] = (m::fma(T(-2), k2[j], k1[j]) + k3[j]) * T(1.0 / 6.0);
}

// Rodas4 and Rodas5P (Sec. 5.2.1: GPURodas4 after Hairer-Wanner, GPURodas5P after
// Steinebach 2023): stiffly accurate Rosenbrock methods of orders 4(3) and 5(4), in the
// transformed form the publications give their coefficients in.  With W = I - h gamma J and
// stages U_i (i = 0..S-1):
//   W U_i = h gamma f(y + sum_{j<i} a_ij U_j) + gamma sum_{j<i} c_ij U_j,
//   y_{n+1} = (the last stage's argument) + U_{S-1},   E = U_{S-1}
// (the last stage's argument is the embedded solution).  Autonomous models: the stage times
// and the time-derivative terms do not enter.
struct Rodas4Tab {
  static constexpr int S = 6;
  static constexpr double gamma = 0.25;
  // stage 5's argument adds U_4 to stage 4's
  static __host__ __device__ constexpr double a(int i, int j) {
    constexpr double v[6][5] = {
        {0, 0, 0, 0, 0},
        {1.544, 0, 0, 0, 0},
        {0.9466785280815826, 0.2557011698983284, 0, 0, 0},
        {3.314825187068521, 2.896124015972201, 0.9986419139977817, 0, 0},
        {1.221224509226641, 6.019134481288629, 12.53708332932087, -0.6878860361058950, 0},
        {1.221224509226641, 6.019134481288629, 12.53708332932087, -0.6878860361058950, 1.0}};
    return v[i][j];
  }
  static __host__ __device__ constexpr double c(int i, int j) {
    constexpr double v[6][5] = {
        {0, 0, 0, 0, 0},
        {-5.6688, 0, 0, 0, 0},
        {-2.430093356833875, -0.2063599157091915, 0, 0, 0},
        {-0.1073529058151375, -9.594562251023355, -20.47028614809616, 0, 0},
        {7.496443313967647, -10.24680431464352, -33.99990352819905, 11.70890893206160, 0},
        {8.083246795921522, -7.981132988064893, -31.52159432874371, 16.31930543123136,
         -6.058818238834054}};
    return v[i][j];
  }
};

struct Rodas5PTab {
  static constexpr int S = 8;
  static constexpr double gamma = 0.21193756319429014;
  // stages 6 and 7 each add the previous stage's U to the argument before them
  static __host__ __device__ constexpr double a(int i, int j) {
    constexpr double v[8][7] = {
        {0, 0, 0, 0, 0, 0, 0},
        {3.0, 0, 0, 0, 0, 0, 0},
        {2.849394379747939, 0.45842242204463923, 0, 0, 0, 0, 0},
        {-6.954028509809101, 2.489845061869568, -10.358996098473584, 0, 0, 0, 0},
        {2.8029986275628964, 0.5072464736228206, -0.3988312541770524, -0.04721187230404641, 0, 0,
         0},
        {-7.502846399306121, 2.561846144803919, -11.627539656261098, -0.18268767659942256,
         0.030198172008377946, 0, 0},
        {-7.502846399306121, 2.561846144803919, -11.627539656261098, -0.18268767659942256,
         0.030198172008377946, 1.0, 0},
        {-7.502846399306121, 2.561846144803919, -11.627539656261098, -0.18268767659942256,
         0.030198172008377946, 1.0, 1.0}};
    return v[i][j];
  }
  static __host__ __device__ constexpr double c(int i, int j) {
    constexpr double v[8][7] = {
        {0, 0, 0, 0, 0, 0, 0},
        {-14.155112264123755, 0, 0, 0, 0, 0, 0},
        {-17.97296035885952, -2.859693295451294, 0, 0, 0, 0, 0},
        {147.12150275711716, -1.41221402718213, 71.68940251302358, 0, 0, 0, 0},
        {165.43517024871676, -0.4592823456491126, 42.90938336958603, -5.961986721573306, 0, 0,
         0},
        {24.854864614690072, -3.0009227002832186, 47.4931110020768, 5.5814197821558125,
         -0.6610691825249471, 0, 0},
        {30.91273214028599, -3.1208243349937974, 77.79954646070892, 34.28646028294783,
         -19.097331116725623, -28.087943162872662, 0},
        {37.80277123390563, -3.2571969029072276, 112.26918849496327, 66.9347231244047,
         -40.06618937091002, -54.66780262877968, -9.48861652309627}};
    return v[i][j];
  }
};

// One Rodas step from (u, t) with f0 = f(u, t): fills unew = y_{n+1}, err = E (the full error,
// not divided by h) and f1 = f(unew) (the next step's f0).
template <class RHS, class T, class TAB>
__device__ __forceinline__ void rodas_step(const T* u, const T* p, T t, T h, const T* f0,
                                           T* unew, T* err, T* f1) {
  static_assert(RHS::autonomous, "the Rodas methods here assume df/dt = 0");
  constexpr int D = RHS::D, S = TAB::S;
  typedef M<T> m;
  const T hg = h * T(TAB::gamma);
  RosLUOf<RHS, T> lu;
  ros_factor<RHS, T>(u, p, t, hg, lu);
  T U[S][D], g[D], fi[D], v[D];
#pragma unroll
  for (int i = 0; i < S; ++i) {
    if (i == 0) {
#pragma unroll
      for (int j = 0; j < D; ++j) v[j] = hg * f0[j];
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        T x = u[j];
#pragma unroll
        for (int l = 0; l < i; ++l) x = m::fma(T(TAB::a(i, l)), U[l][j], x);
        g[j] = x;
      }
      RHS::f(g, p, t, fi);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        T x = hg * fi[j];
#pragma unroll
        for (int l = 0; l < i; ++l) x = m::fma(T(TAB::gamma * TAB::c(i, l)), U[l][j], x);
        v[j] = x;
      }
    }
    lu.solve(v, U[i]);
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    unew[j] = g[j] + U[S - 1][j];
    err[j] = U[S - 1][j];
  }
  RHS::f(unew, p, t + h, f1);
}

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
struct Philox {
  static __device__ __forceinline__ uint4 gen(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      if (r > 0) {
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
      }
      const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
      const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
      c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
  }
  static __device__ __forceinline__ uint4 call(unsigned long long seed, unsigned long long traj,
                                               unsigned long long idx) {
    return gen(make_uint4(uint32_t(idx), uint32_t(idx >> 32), uint32_t(traj),
                          uint32_t(traj >> 32)),
               make_uint2(uint32_t(seed), uint32_t(seed >> 32)));
  }
};

// Normals from one Philox call: 4 in FP32, 2 in FP64 (Box-Muller of exact uniforms).
template <class T>
struct Normals;

template <>
struct Normals<float> {
  static constexpr int per_call = 4;
  static __device__ __forceinline__ float uni(uint32_t x) {
    // ((x >> 9) + 0.5) * 2^-23, exact and inside (0, 1), without an integer conversion: the
    // bits 1.m (m = x >> 9) are 1 + m 2^-23, and subtracting 1 - 2^-24 is exact (Sterbenz)
    return __int_as_float(0x3F800000u | (x >> 9)) - 0.99999994039535522f;
  }
  static __device__ __forceinline__ void draw(uint4 x, float* z) {
    float s, c;
    // log and sincospi stay the accurate library functions (the MUFU log loses relative
    // accuracy as u -> 1); the radius square root is the MUFU one (~1 ulp)
    float r = M<float>::fast_sqrt(-2.0f * logf(uni(x.x)));
    sincospif(2.0f * uni(x.y), &s, &c);
    z[0] = r * c;
    z[1] = r * s;
    r = M<float>::fast_sqrt(-2.0f * logf(uni(x.z)));
    sincospif(2.0f * uni(x.w), &s, &c);
    z[2] = r * c;
    z[3] = r * s;
  }
};

template <>
struct Normals<double> {
  static constexpr int per_call = 2;
  static __device__ __forceinline__ double uni(uint32_t hi, uint32_t lo) {
    const unsigned long long v = ((unsigned long long)hi << 32) | lo;
    // ((v >> 12) + 0.5) * 2^-52: exact in double, inside (0, 1)
    return __fma_rn(__ull2double_rn(v >> 12), 2.220446049250313e-16, 1.1102230246251565e-16);
  }
  static __device__ __forceinline__ void draw(uint4 x, double* z) {
    double s, c;
    const double r = ::sqrt(-2.0 * ::log(uni(x.x, x.y)));
    sincospi(2.0 * uni(x.z, x.w), &s, &c);
    z[0] = r * c;
    z[1] = r * s;
  }
};

}  // namespace ens
