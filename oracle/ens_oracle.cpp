// ens_oracle.cpp -- plain, slow, obviously-correct CPU oracle for the ensemble solver.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this file;
// only tests/, the smoke check in __graft_entry__ and bench.py's CPU-baseline / reference
// legs use it.  It shares no source, header, table or constant with the CUDA path.
//
// What it computes (arXiv 2304.06835, "Automated Translation and Accelerated Solving of
// Differential Equations on Multiple GPU Platforms"):
//   * the ensemble problem: N independent copies of du/dt = f(u,p,t), one (p_j, u0_j, tspan_j)
//     per trajectory (Sec. 5.1.1, the U / P / F matrices);
//   * explicit Runge-Kutta steps from a tableau {A,b,c} (Sec. 3.1, the k_s / u_{n+1} equations),
//     here Tsitouras' 5(4) pair (GPUTsit5, Sec. 5.2.1) and the classic RK4;
//   * the embedded error estimate, the scaled error ratio q and PI step control
//     (Sec. 3.1, the q equation and h_new = eta q_{n-1}^{beta2} q_n^{beta1} h);
//   * the Rosenbrock method (Sec. 3.2.1, the s-stage Rosenbrock formulas), as the
//     Shampine-Reichelt order-2(3) Rosenbrock-W pair named by GPURosenbrock23 (Sec. 5.2.1);
//   * Euler-Maruyama for dX = a dt + b dW, dW ~ N(0,dt) (Sec. 3.3, the SDE definition; GPUEM);
//   * the benchmark models: Lorenz (Appendix, Lorenz problem), Robertson (Appendix, Robertson
//     equation) and the linear asset-price SDE / geometric Brownian motion (Appendix, linear SDE).
//
// Readings where the paper is silent (every one is listed in the design notes):
//   * Tsit5 coefficients: Tsitouras (2011), Comput. Math. Appl. 62, table of the 5(4) pair.
//   * error norm: root-mean-square over the D components (Hairer-Norsett-Wanner I, II.4).
//   * accept iff q <= 1;  PI constants eta=0.9, beta1=0.7/k, beta2=0.4/k (k=5 Tsit5, k=3 R23),
//     fac clamped to [0.2,10], reject factor max(0.2, eta q^{-1/k}), q_{n-1} starts at 1e-4 and is
//     max(q,1e-4) after an accept, q guarded below by 1e-10.
//   * automatic first step: Hairer-Norsett-Wanner I, II.4 starting step size algorithm.
//   * Rosenbrock23: d = 1/(2+sqrt2), e32 = 6+sqrt2 (Shampine & Reichelt 1997, ode23s).
//   * random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = seed,
//     counter = (draw index lo, hi, trajectory index lo, hi); uniforms ((x>>9)+0.5)*2^-23 (FP32)
//     or ((x0:x1 >> 12)+0.5)*2^-52 (FP64), both exact and inside (0,1); Box-Muller normals.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared -pthread (see oracle/__init__.py).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

// ----------------------------------------------------------------------------------------------
// identifiers (values match the public C-ABI enumeration by documentation, not by a shared header)
enum {
  RHS_LORENZ = 1, RHS_ROBERTSON = 2, RHS_GBM = 3, RHS_CRN = 4, RHS_BALL = 5,
  RHS_OREGO = 6, RHS_HIRES = 7, RHS_POLLU = 8
};
enum {
  ALG_TSIT5_FIXED = 1, ALG_TSIT5_ADAPTIVE = 2, ALG_RK4 = 3, ALG_ROS23 = 4, ALG_EM = 5,
  ALG_RODAS4 = 6, ALG_RODAS5P = 7, ALG_SIEA = 8
};
enum { ST_OK = 0, ST_MAXITERS = 1, ST_DT_MIN = 2, ST_NONFINITE = 3 };
enum { LAYOUT_ROWMAJOR = 0, LAYOUT_SOA = 1 };
constexpr int MAXD = 20, MAXP = 25;  // largest model: POLLU (D = 20, P = 25)

// ----------------------------------------------------------------------------------------------
// Models (Appendix: Lorenz, Robertson, linear SDE, sigma-factor CRN).  f(u,p,t), the
// diffusion matrix of the SDE models and the Jacobians df/du, df/dp of the ODE models.
// Mw = number of Wiener processes (0 for an ODE).
struct Model {
  int D, P, Mw;
};

Model model_of(int rhs) {
  switch (rhs) {
    case RHS_LORENZ: return {3, 3, 0};
    case RHS_ROBERTSON: return {3, 3, 0};
    case RHS_GBM: return {1, 2, 1};
    case RHS_CRN: return {4, 6, 8};
    case RHS_BALL: return {2, 2, 0};
    case RHS_OREGO: return {3, 3, 0};
    case RHS_HIRES: return {8, 12, 0};
    case RHS_POLLU: return {20, 25, 0};
  }
  return {0, 0, 0};
}

// Lorenz: p = (sigma, rho, beta); the paper writes beta as gamma.
template <class T>
void f_lorenz(const T* u, const T* p, T /*t*/, T* du) {
  const T sigma = p[0], rho = p[1], beta = p[2];
  du[0] = sigma * (u[1] - u[0]);
  du[1] = rho * u[0] - u[1] - u[0] * u[2];
  du[2] = u[0] * u[1] - beta * u[2];
}

// Robertson: p = (k1, k2, k3) with k1 on y1, k2 on y2^2, k3 on y2*y3.
template <class T>
void f_robertson(const T* u, const T* p, T /*t*/, T* du) {
  const T k1 = p[0], k2 = p[1], k3 = p[2];
  du[0] = -k1 * u[0] + k3 * u[1] * u[2];
  du[1] = k1 * u[0] - k3 * u[1] * u[2] - k2 * u[1] * u[1];
  du[2] = k2 * u[1] * u[1];
}

// Geometric Brownian motion drift a(X) = mu X (diffusion b(X) = sigma X below); p = (mu, sigma).
template <class T>
void f_gbm(const T* u, const T* p, T /*t*/, T* du) {
  du[0] = p[0] * u[0];
}

template <class T>
void g_gbm(const T* u, const T* p, T /*t*/, T* gu) {
  gu[0] = p[1] * u[0];
}

// Sigma-factor stress-response CRN (Appendix, SDE models), the Chemical Langevin form with
// 4 species u = ([sigma], [A1], [A2], [A3]) and p = (S, D, tau, nu0, n, eta).
// Drift:   d[sigma] = nu0 + H - [sigma],  H = (S[sigma])^n / ((S[sigma])^n + (D[A3])^n + 1),
//          d[A1] = [sigma]/tau - [A1]/tau,  d[A2] = [A1]/tau - [A2]/tau,
//          d[A3] = [A2]/tau - [A3]/tau.
// Noise (8 Wiener processes, column m of G multiplies dW_{m+1}):
//          [sigma]: +eta sqrt(nu0 + H) dW1 - eta sqrt([sigma]) dW2,
//          [A1]:    +eta sqrt([sigma]/tau) dW3 - eta sqrt([A1]/tau) dW4,
//          [A2]:    +eta sqrt([A1]/tau) dW5 - eta sqrt([A2]/tau) dW6,
//          [A3]:    +eta sqrt([A2]/tau) dW7 - eta sqrt([A3]/tau) dW8.
// The Langevin form is defined for non-negative amounts; a path of it can step below zero, so
// every square-root argument and both Hill bases are taken as max(., 0).
template <class T>
T crn_hill(const T* u, const T* p) {
  const T a = std::pow(std::max(p[0] * u[0], T(0)), p[4]);
  const T b = std::pow(std::max(p[1] * u[3], T(0)), p[4]);
  return a / (a + b + T(1));
}

template <class T>
void f_crn(const T* u, const T* p, T /*t*/, T* du) {
  const T tau = p[2], nu0 = p[3];
  du[0] = nu0 + crn_hill(u, p) - u[0];
  du[1] = u[0] / tau - u[1] / tau;
  du[2] = u[1] / tau - u[2] / tau;
  du[3] = u[2] / tau - u[3] / tau;
}

template <class T>
T sqrt0(T x) {
  return std::sqrt(std::max(x, T(0)));
}

// G[j*8 + m] = coefficient of dW_{m+1} in the equation of species j
template <class T>
void g_crn(const T* u, const T* p, T /*t*/, T* G) {
  const T tau = p[2], nu0 = p[3], eta = p[5];
  for (int i = 0; i < 32; ++i) G[i] = T(0);
  G[0 * 8 + 0] = eta * sqrt0(nu0 + crn_hill(u, p));
  G[0 * 8 + 1] = -eta * sqrt0(u[0]);
  G[1 * 8 + 2] = eta * sqrt0(u[0] / tau);
  G[1 * 8 + 3] = -eta * sqrt0(u[1] / tau);
  G[2 * 8 + 4] = eta * sqrt0(u[1] / tau);
  G[2 * 8 + 5] = -eta * sqrt0(u[2] / tau);
  G[3 * 8 + 6] = eta * sqrt0(u[2] / tau);
  G[3 * 8 + 7] = -eta * sqrt0(u[3] / tau);
}

// diffusion matrix G [D][Mw] of an SDE model
template <class T>
void diffusion(int id, const T* u, const T* p, T t, T* G) {
  if (id == RHS_GBM) g_gbm(u, p, t, G);
  else g_crn(u, p, t, G);
}

// Bouncing ball (Sec. 6.5 event handling; Appendix, bouncing-ball problem): u = (x, v),
// p = (g, e); dx/dt = v, dv/dt = -g.  Event: the condition x = 0 reached from above
// triggers the affect v <- -e v (e the coefficient of restitution).
template <class T>
void f_ball(const T* u, const T* p, T /*t*/, T* du) {
  du[0] = u[1];
  du[1] = -p[0];
}

bool has_event(int id) { return id == RHS_BALL; }

// Oregonator (Appendix, OREGO): p = (k1, k2, k3).  The first equation's leading sign is read
// as + (the Field-Noyes model the paper cites): with the printed minus the concentrations
// run to -infinity from the printed initial state.
template <class T>
void f_orego(const T* y, const T* k, T /*t*/, T* dy) {
  dy[0] = k[0] * (y[1] + y[0] * (1 - k[1] * y[0] - y[1]));
  dy[1] = (y[2] - (1 + y[0]) * y[1]) / k[0];
  dy[2] = k[2] * (y[0] - y[2]);
}

// HIRES (Appendix): the distinct rate constants as p = (c1..c12) =
// (1.71, 0.43, 8.32, 0.0007, 8.75, 10.03, 0.035, 1.12, 1.745, 280.0, 0.69, 1.81);
// a constant printed in several equations is the same parameter in each.
template <class T>
void f_hires(const T* y, const T* c, T /*t*/, T* dy) {
  dy[0] = -c[0] * y[0] + c[1] * y[1] + c[2] * y[2] + c[3];
  dy[1] = c[0] * y[0] - c[4] * y[1];
  dy[2] = -c[5] * y[2] + c[1] * y[3] + c[6] * y[4];
  dy[3] = c[2] * y[1] + c[0] * y[2] - c[7] * y[3];
  dy[4] = -c[8] * y[4] + c[1] * y[5] + c[1] * y[6];
  dy[5] = -c[9] * y[5] * y[7] + c[10] * y[3] + c[0] * y[4] - c[1] * y[5] + c[10] * y[6];
  dy[6] = c[9] * y[5] * y[7] - c[11] * y[6];
  dy[7] = -c[9] * y[5] * y[7] + c[11] * y[6];
}

// POLLU (Appendix): p = (k1..k25), the printed equations term by term (the printed "k7 u9"
// and "2 k18 u16" read as k7 y9 and 2 k18 y16).  0-based: y[i] is y_{i+1}, k[j] is k_{j+1}.
template <class T>
void f_pollu(const T* y, const T* k, T /*t*/, T* dy) {
  dy[0] = -k[0] * y[0] - k[9] * y[10] * y[0] - k[13] * y[0] * y[5] - k[22] * y[0] * y[3] -
          k[23] * y[18] * y[0] + k[1] * y[1] * y[3] + k[2] * y[4] * y[1] + k[8] * y[10] * y[1] +
          k[10] * y[12] + k[11] * y[9] * y[1] + k[21] * y[18] + k[24] * y[19];
  dy[1] = -k[1] * y[1] * y[3] - k[2] * y[4] * y[1] - k[8] * y[10] * y[1] -
          k[11] * y[9] * y[1] + k[0] * y[0] + k[20] * y[18];
  dy[2] = -k[14] * y[2] + k[0] * y[0] + k[16] * y[3] + k[18] * y[15] + k[21] * y[18];
  dy[3] = -k[1] * y[1] * y[3] - k[15] * y[3] - k[16] * y[3] - k[22] * y[0] * y[3] +
          k[14] * y[2];
  dy[4] = -k[2] * y[4] * y[1] + 2 * k[3] * y[6] + k[5] * y[6] * y[5] + k[6] * y[8] +
          k[12] * y[13] + k[19] * y[16] * y[5];
  dy[5] = -k[5] * y[6] * y[5] - k[7] * y[8] * y[5] - k[13] * y[0] * y[5] -
          k[19] * y[16] * y[5] + k[2] * y[4] * y[1] + 2 * k[17] * y[15];
  dy[6] = -k[3] * y[6] - k[4] * y[6] - k[5] * y[6] * y[5] + k[12] * y[13];
  dy[7] = k[3] * y[6] + k[4] * y[6] + k[5] * y[6] * y[5] + k[6] * y[8];
  dy[8] = -k[6] * y[8] - k[7] * y[8] * y[5];
  dy[9] = -k[11] * y[9] * y[1] + k[6] * y[8] + k[8] * y[10] * y[1];
  dy[10] = -k[8] * y[10] * y[1] - k[9] * y[10] * y[0] + k[7] * y[8] * y[5] + k[10] * y[12];
  dy[11] = k[8] * y[10] * y[1];
  dy[12] = -k[10] * y[12] + k[9] * y[10] * y[0];
  dy[13] = -k[12] * y[13] + k[11] * y[9] * y[1];
  dy[14] = k[13] * y[0] * y[5];
  dy[15] = -k[17] * y[15] - k[18] * y[15] + k[15] * y[3];
  dy[16] = -k[19] * y[16] * y[5];
  dy[17] = k[19] * y[16] * y[5];
  dy[18] = -k[20] * y[18] - k[21] * y[18] - k[23] * y[18] * y[0] + k[22] * y[0] * y[3] +
           k[24] * y[19];
  dy[19] = -k[24] * y[19] + k[23] * y[18] * y[0];
}

// POLLU as 25 mass-action reactions: rate r_j = k_j times its reactants, and the change of
// each species per unit of r_j.  The printed equations are exactly sum_j nu_j r_j (tested);
// the Jacobian is sum_j nu_j (d r_j / d y)^T.
struct PolluReaction {
  int a, b;           // reactant indices (b = -1: first order)
  int n;              // number of species changed
  int sp[5];
  double nu[5];
};
const PolluReaction POLLU_R[25] = {
    {0, -1, 3, {0, 1, 2}, {-1, 1, 1}},           // k1:  y1 -> y2 + y3
    {1, 3, 3, {0, 1, 3}, {1, -1, -1}},           // k2:  y2 + y4 -> y1
    {4, 1, 4, {0, 1, 4, 5}, {1, -1, -1, 1}},     // k3:  y5 + y2 -> y1 + y6
    {6, -1, 3, {4, 6, 7}, {2, -1, 1}},           // k4:  y7 -> 2 y5 + y8
    {6, -1, 2, {6, 7}, {-1, 1}},                 // k5:  y7 -> y8
    {6, 5, 4, {4, 5, 6, 7}, {1, -1, -1, 1}},     // k6:  y7 + y6 -> y5 + y8
    {8, -1, 4, {4, 7, 8, 9}, {1, 1, -1, 1}},     // k7:  y9 -> y5 + y8 + y10
    {8, 5, 3, {5, 8, 10}, {-1, -1, 1}},          // k8:  y9 + y6 -> y11
    {10, 1, 5, {0, 1, 9, 10, 11}, {1, -1, 1, -1, 1}},  // k9: y11 + y2 -> y1 + y10 + y12
    {10, 0, 3, {0, 10, 12}, {-1, -1, 1}},        // k10: y11 + y1 -> y13
    {12, -1, 3, {0, 10, 12}, {1, 1, -1}},        // k11: y13 -> y1 + y11
    {9, 1, 4, {0, 1, 9, 13}, {1, -1, -1, 1}},    // k12: y10 + y2 -> y1 + y14
    {13, -1, 3, {4, 6, 13}, {1, 1, -1}},         // k13: y14 -> y5 + y7
    {0, 5, 3, {0, 5, 14}, {-1, -1, 1}},          // k14: y1 + y6 -> y15
    {2, -1, 2, {2, 3}, {-1, 1}},                 // k15: y3 -> y4
    {3, -1, 2, {3, 15}, {-1, 1}},                // k16: y4 -> y16
    {3, -1, 2, {2, 3}, {1, -1}},                 // k17: y4 -> y3
    {15, -1, 2, {5, 15}, {2, -1}},               // k18: y16 -> 2 y6
    {15, -1, 2, {2, 15}, {1, -1}},               // k19: y16 -> y3
    {16, 5, 4, {4, 5, 16, 17}, {1, -1, -1, 1}},  // k20: y17 + y6 -> y5 + y18
    {18, -1, 2, {1, 18}, {1, -1}},               // k21: y19 -> y2
    {18, -1, 3, {0, 2, 18}, {1, 1, -1}},         // k22: y19 -> y1 + y3
    {0, 3, 3, {0, 3, 18}, {-1, -1, 1}},          // k23: y1 + y4 -> y19
    {18, 0, 3, {0, 18, 19}, {-1, -1, 1}},        // k24: y19 + y1 -> y20
    {19, -1, 3, {0, 18, 19}, {1, 1, -1}},        // k25: y20 -> y1 + y19
};

template <class T>
void jac_stiff(int id, const T* y, const T* k, T* J) {
  const int D = id == RHS_OREGO ? 3 : id == RHS_HIRES ? 8 : 20;
  for (int i = 0; i < D * D; ++i) J[i] = 0;
  if (id == RHS_OREGO) {
    J[0] = k[0] * (1 - 2 * k[1] * y[0] - y[1]);
    J[1] = k[0] * (1 - y[0]);
    J[3] = -y[1] / k[0];
    J[4] = -(1 + y[0]) / k[0];
    J[5] = 1 / k[0];
    J[6] = k[2];
    J[8] = -k[2];
  } else if (id == RHS_HIRES) {
    const T* c = k;
    auto at = [&](int i, int j) -> T& { return J[i * 8 + j]; };
    at(0, 0) = -c[0]; at(0, 1) = c[1]; at(0, 2) = c[2];
    at(1, 0) = c[0]; at(1, 1) = -c[4];
    at(2, 2) = -c[5]; at(2, 3) = c[1]; at(2, 4) = c[6];
    at(3, 1) = c[2]; at(3, 2) = c[0]; at(3, 3) = -c[7];
    at(4, 4) = -c[8]; at(4, 5) = c[1]; at(4, 6) = c[1];
    at(5, 3) = c[10]; at(5, 4) = c[0]; at(5, 5) = -c[9] * y[7] - c[1]; at(5, 6) = c[10];
    at(5, 7) = -c[9] * y[5];
    at(6, 5) = c[9] * y[7]; at(6, 6) = -c[11]; at(6, 7) = c[9] * y[5];
    at(7, 5) = -c[9] * y[7]; at(7, 6) = c[11]; at(7, 7) = -c[9] * y[5];
  } else {  // POLLU: sum over the reactions of nu_j (d r_j / d y)^T
    for (int j = 0; j < 25; ++j) {
      const PolluReaction& r = POLLU_R[j];
      const T dra = r.b < 0 ? k[j] : k[j] * y[r.b];  // d r_j / d y_a
      const T drb = r.b < 0 ? T(0) : k[j] * y[r.a];  // d r_j / d y_b
      for (int m = 0; m < r.n; ++m) {
        J[r.sp[m] * 20 + r.a] += T(r.nu[m]) * dra;
        if (r.b >= 0) J[r.sp[m] * 20 + r.b] += T(r.nu[m]) * drb;
      }
    }
  }
}

// POLLU's right-hand side as the reaction sum (for the test that it equals the printed form)
void pollu_reaction_sum(const double* y, const double* k, double* dy) {
  for (int i = 0; i < 20; ++i) dy[i] = 0;
  for (int j = 0; j < 25; ++j) {
    const PolluReaction& r = POLLU_R[j];
    const double rate = k[j] * y[r.a] * (r.b < 0 ? 1.0 : y[r.b]);
    for (int m = 0; m < r.n; ++m) dy[r.sp[m]] += r.nu[m] * rate;
  }
}

template <class T>
T event_condition(int /*id*/, const T* u, const T* /*p*/, T /*t*/) {
  return u[0];
}

template <class T>
void event_affect(int /*id*/, T* u, const T* p, T /*t*/) {
  u[1] = -p[1] * u[1];
}

template <class T>
void rhs(int id, const T* u, const T* p, T t, T* du) {
  if (id == RHS_LORENZ) f_lorenz(u, p, t, du);
  else if (id == RHS_ROBERTSON) f_robertson(u, p, t, du);
  else if (id == RHS_GBM) f_gbm(u, p, t, du);
  else if (id == RHS_CRN) f_crn(u, p, t, du);
  else if (id == RHS_BALL) f_ball(u, p, t, du);
  else if (id == RHS_OREGO) f_orego(u, p, t, du);
  else if (id == RHS_HIRES) f_hires(u, p, t, du);
  else f_pollu(u, p, t, du);
}

// J[i*D+j] = d f_i / d u_j
// df/du of the stiff models OREGO, HIRES, POLLU (defined with them below)
template <class T>
void jac_stiff(int id, const T* u, const T* p, T* J);

template <class T>
void jac_u(int id, const T* u, const T* p, T /*t*/, T* J) {
  if (id == RHS_LORENZ) {
    const T sigma = p[0], rho = p[1], beta = p[2];
    J[0] = -sigma; J[1] = sigma; J[2] = 0;
    J[3] = rho - u[2]; J[4] = -1; J[5] = -u[0];
    J[6] = u[1]; J[7] = u[0]; J[8] = -beta;
  } else if (id == RHS_ROBERTSON) {
    const T k1 = p[0], k2 = p[1], k3 = p[2];
    J[0] = -k1; J[1] = k3 * u[2]; J[2] = k3 * u[1];
    J[3] = k1; J[4] = -k3 * u[2] - 2 * k2 * u[1]; J[5] = -k3 * u[1];
    J[6] = 0; J[7] = 2 * k2 * u[1]; J[8] = 0;
  } else if (id == RHS_GBM) {
    J[0] = p[0];
  } else {
    jac_stiff<T>(id, u, p, J);
  }
}

// Jp[i*P+m] = d f_i / d p_m
template <class T>
void jac_p(int id, const T* u, const T* /*p*/, T /*t*/, T* Jp) {
  if (id == RHS_LORENZ) {
    Jp[0] = u[1] - u[0]; Jp[1] = 0; Jp[2] = 0;
    Jp[3] = 0; Jp[4] = u[0]; Jp[5] = 0;
    Jp[6] = 0; Jp[7] = 0; Jp[8] = -u[2];
  } else if (id == RHS_ROBERTSON) {
    Jp[0] = -u[0]; Jp[1] = 0; Jp[2] = u[1] * u[2];
    Jp[3] = u[0]; Jp[4] = -u[1] * u[1]; Jp[5] = -u[1] * u[2];
    Jp[6] = 0; Jp[7] = u[1] * u[1]; Jp[8] = 0;
  } else {
    Jp[0] = u[0]; Jp[1] = 0;
  }
}

// ----------------------------------------------------------------------------------------------
// Tsitouras 5(4) tableau (Tsitouras 2011).  Stage 7 is the FSAL stage: row 7 of A equals b.
// bhat is the embedded 4th-order weight vector; the error estimate is h * sum (b_i - bhat_i) k_i.
const double TS_C[7] = {0.0, 0.161, 0.327, 0.9, 0.9800255409045097, 1.0, 1.0};
const double TS_A[7][7] = {
    {0, 0, 0, 0, 0, 0, 0},
    {0.161, 0, 0, 0, 0, 0, 0},
    {-0.008480655492356989, 0.335480655492357, 0, 0, 0, 0, 0},
    {2.897153057105493, -6.359448489975075, 4.3622954328695815, 0, 0, 0, 0},
    {5.325864828439257, -11.748883564062828, 7.4955393428898365, -0.09249506636175525, 0, 0, 0},
    {5.86145544294642, -12.92096931784711, 8.159367898576159, -0.071584973281401,
     -0.028269050394068383, 0, 0},
    {0.09646076681806523, 0.01, 0.4798896504144996, 1.379008574103742, -3.290069515436081,
     2.324710524099774, 0},
};
const double TS_B[7] = {0.09646076681806523, 0.01, 0.4798896504144996, 1.379008574103742,
                        -3.290069515436081, 2.324710524099774, 0.0};
const double TS_BHAT[7] = {0.09468075576583945, 0.009183565540343254, 0.4877705284247616,
                           1.234297566930479, -2.7077123499835256, 1.866628418170587,
                           0.015151515151515152};

// Controller constants (readings listed in the file header).
const double ETA = 0.9;
const double FAC_MIN = 0.2, FAC_MAX = 10.0;
const double QOLD_INIT = 1e-4, Q_FLOOR = 1e-10;

template <class T>
struct Prec;
template <>
struct Prec<double> {
  static constexpr double dtmin_factor = 1e-14;
};
template <>
struct Prec<float> {
  static constexpr double dtmin_factor = 1e-9;
};
const double STOP_EPS = 1e-12;  // a remainder this small (relative) counts as having arrived

// ----------------------------------------------------------------------------------------------
// Time accumulator.  FP64: plain sum.  FP32: Neumaier-compensated (t = hi + lo).
template <class T>
struct Clock {
  T hi, lo;
  void set(T v) { hi = v; lo = 0; }
  T value() const { return hi + lo; }
  T remaining(T stop) const { return (stop - hi) - lo; }
  void add(T h) {
    T s = hi + h;
    if (std::fabs(hi) >= std::fabs(h)) lo += (hi - s) + h;
    else lo += (h - s) + hi;
    hi = s;
  }
};
template <>
struct Clock<double> {
  double hi;
  void set(double v) { hi = v; }
  double value() const { return hi; }
  double remaining(double stop) const { return stop - hi; }
  void add(double h) { hi += h; }
};

template <class T>
bool finite_all(const T* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// scaled RMS norm  sqrt( (1/D) sum_j (x_j / sc_j)^2 )
template <class T>
T rms_scaled(const T* x, const T* sc, int D) {
  T s = 0;
  for (int j = 0; j < D; ++j) {
    T r = x[j] / sc[j];
    s += r * r;
  }
  return std::sqrt(s / T(D));
}

// ----------------------------------------------------------------------------------------------
// One Tsit5 step of size h from (u,t) with k1 = f(u,t) given.  Fills unew, err (= h sum btilde k),
// k7 = f(unew, t+h).  Stage formula: U_i = u + h sum_j a_ij k_j, k_i = f(U_i, t + c_i h).
template <class T>
void tsit5_step(int id, int D, const T* u, const T* p, T t, T h, const T* k1, T* unew, T* err,
                T* k7, T (*kout)[MAXD] = nullptr) {
  T k[7][MAXD];
  T U[MAXD];
  for (int j = 0; j < D; ++j) k[0][j] = k1[j];
  for (int i = 1; i < 7; ++i) {
    for (int j = 0; j < D; ++j) {
      T s = 0;
      for (int m = 0; m < i; ++m) s += T(TS_A[i][m]) * k[m][j];
      U[j] = u[j] + h * s;
    }
    rhs<T>(id, U, p, t + T(TS_C[i]) * h, k[i]);
  }
  // u_{n+1} = u_n + h sum b_i k_i  (b_7 = 0)
  for (int j = 0; j < D; ++j) {
    T s = 0;
    for (int m = 0; m < 7; ++m) s += T(TS_B[m]) * k[m][j];
    unew[j] = u[j] + h * s;
  }
  // E = u~ - u_{n+1} = h sum (bhat_i - b_i) k_i
  for (int j = 0; j < D; ++j) {
    T s = 0;
    for (int m = 0; m < 7; ++m) s += T(TS_BHAT[m] - TS_B[m]) * k[m][j];
    err[j] = h * s;
    k7[j] = k[6][j];
  }
  if (kout)
    for (int i = 0; i < 7; ++i)
      for (int j = 0; j < D; ++j) kout[i][j] = k[i][j];
}

// Dense output of a Tsit5 step: u(t_n + theta h) = u_n + h sum_i b_i(theta) k_i with
// b_i(theta) = sum_q TS_DENSE[i][q] theta^(q+1).  TS_DENSE is the continuous extension of
// order 4 defined by the order conditions of the trees of order <= 4 at every theta,
// b_i(1) = b_i and C1 continuity, with the one free parameter minimising the integrated
// 5th-order defect (values from oracle/dense.py, which derives them in 40 digits).
const double TS_DENSE[7][4] = {
    {1.0, -2.7697190760997743, 2.925281219471809, -1.0591013765539699},
    {0.0, 0.12894208371183252, -0.2178841674236653, 0.09894208371183272},
    {0.0, 3.956917849412212, -5.994277097166426, 2.5172488981687136},
    {0.0, -12.899911070336683, 31.315856437088335, -17.03693679264791},
    {0.0, 39.47651640903875, -92.11331087982184, 49.346724955347},
    {0.0, -29.443928026595056, 68.1866981495892, -36.418059598894374},
    {0.0, 1.5511818308687129, -4.102363661737424, 2.551181830868712}};

template <class T>
void tsit5_dense(int D, const T* u, T h, const T (*k)[MAXD], T theta, T* out) {
  T bw[7];
  for (int i = 0; i < 7; ++i)
    bw[i] = theta * (T(TS_DENSE[i][0]) +
                     theta * (T(TS_DENSE[i][1]) +
                              theta * (T(TS_DENSE[i][2]) + theta * T(TS_DENSE[i][3]))));
  for (int j = 0; j < D; ++j) {
    T s = 0;
    for (int i = 0; i < 7; ++i) s += bw[i] * k[i][j];
    out[j] = u[j] + h * s;
  }
}

// ---- events (Sec. 6.5): a condition g(u, p, t) crossing zero from above inside an accepted
// Tsit5 step triggers the model's affect.  The step's dense output is written as a
// polynomial in theta, u(theta) = u_n + sum_{q=1..4} theta^q c_q with c_q = h sum_i r_iq k_i.
// The condition is checked at theta = j / EVENT_POINTS (j = 0..EVENT_POINTS, with u_n and
// u_{n+1} themselves at the ends); the first interval with g > 0 at its left end and g <= 0
// at its right end is narrowed by the Illinois method (regula falsi that halves the value
// kept at an end which survives two iterations in a row; Dowell & Jarratt 1971) until it is
// at most 4 eps wide or after 100 iterations.  The event sits at the interval's right end.
const int EVENT_POINTS = 10;

template <class T>
void dense_coeffs(int D, T h, const T (*k)[MAXD], T (*c)[MAXD]) {
  for (int q = 0; q < 4; ++q)
    for (int j = 0; j < D; ++j) {
      T s = 0;
      for (int i = 0; i < 7; ++i) s += T(TS_DENSE[i][q]) * k[i][j];
      c[q][j] = h * s;
    }
}

template <class T>
void dense_poly(int D, const T* u, const T (*c)[MAXD], T th, T* out) {
  for (int j = 0; j < D; ++j)
    out[j] = u[j] + th * (c[0][j] + th * (c[1][j] + th * (c[2][j] + th * c[3][j])));
}

// theta in (0, 1] of the first crossing from above in the step, or -1 for none
template <class T>
T find_event(int id, int D, const T* u, const T* unew, const T* p, T tn, T h,
             const T (*c)[MAXD]) {
  T w[MAXD];
  auto g_at = [&](T th) {
    dense_poly<T>(D, u, c, th, w);
    return event_condition<T>(id, w, p, tn + th * h);
  };
  T a = 0, ga = event_condition<T>(id, u, p, tn);
  for (int j = 1; j <= EVENT_POINTS; ++j) {
    const T b0 = (j == EVENT_POINTS) ? T(1) : T(j) / T(EVENT_POINTS);
    const T gb0 = (j == EVENT_POINTS) ? event_condition<T>(id, unew, p, tn + h) : g_at(b0);
    if (ga > 0 && gb0 <= 0) {
      T b = b0, gb = gb0;
      int side = 0;
      for (int it = 0; it < 100 && b - a > T(4) * std::numeric_limits<T>::epsilon(); ++it) {
        T x = (a * gb - b * ga) / (gb - ga);
        if (!(x > a && x < b)) x = (a + b) / 2;
        const T gx = g_at(x);
        if (gx > 0) {
          a = x;
          ga = gx;
          if (side == 1) gb /= 2;
          side = 1;
        } else {
          b = x;
          gb = gx;
          if (side == -1) ga /= 2;
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

template <class T>
void rk4_step(int id, int D, const T* u, const T* p, T t, T h, T* unew) {
  T k1[MAXD], k2[MAXD], k3[MAXD], k4[MAXD], U[MAXD];
  rhs<T>(id, u, p, t, k1);
  for (int j = 0; j < D; ++j) U[j] = u[j] + (h / 2) * k1[j];
  rhs<T>(id, U, p, t + h / 2, k2);
  for (int j = 0; j < D; ++j) U[j] = u[j] + (h / 2) * k2[j];
  rhs<T>(id, U, p, t + h / 2, k3);
  for (int j = 0; j < D; ++j) U[j] = u[j] + h * k3[j];
  rhs<T>(id, U, p, t + h, k4);
  for (int j = 0; j < D; ++j) unew[j] = u[j] + (h / 6) * (k1[j] + 2 * k2[j] + 2 * k3[j] + k4[j]);
}

// ---- dense LU with partial pivoting (ties -> lowest row index), then forward/back substitution.
template <class T>
void lu_factor(int D, T* W, int* piv) {
  for (int c = 0; c < D; ++c) {
    int best = c;
    for (int r = c + 1; r < D; ++r)
      if (std::fabs(W[r * D + c]) > std::fabs(W[best * D + c])) best = r;
    piv[c] = best;
    if (best != c)
      for (int j = 0; j < D; ++j) std::swap(W[c * D + j], W[best * D + j]);
    for (int r = c + 1; r < D; ++r) {
      W[r * D + c] /= W[c * D + c];
      for (int j = c + 1; j < D; ++j) W[r * D + j] -= W[r * D + c] * W[c * D + j];
    }
  }
}

template <class T>
void lu_solve(int D, const T* LU, const int* piv, const T* b, T* x) {
  T y[MAXD];
  for (int j = 0; j < D; ++j) y[j] = b[j];
  for (int c = 0; c < D; ++c) std::swap(y[c], y[piv[c]]);
  for (int r = 0; r < D; ++r)
    for (int j = 0; j < r; ++j) y[r] -= LU[r * D + j] * y[j];
  for (int r = D - 1; r >= 0; --r) {
    for (int j = r + 1; j < D; ++j) y[r] -= LU[r * D + j] * y[j];
    y[r] /= LU[r * D + r];
  }
  for (int j = 0; j < D; ++j) x[j] = y[j];
}

// One Rosenbrock23 (ode23s) step from (u,t) with f0 = f(u,t).  W = I - h d J.
// Fills unew, err = h/6 (k1 - 2 k2 + k3), f2 = f(unew, t+h).  All models here are autonomous,
// so df/dt = 0 and the h d T terms vanish.
template <class T>
void ros23_step(int id, int D, const T* u, const T* p, T t, T h, const T* f0, T* unew, T* err,
                T* f2) {
  const T d = T(1.0 / (2.0 + std::sqrt(2.0)));
  const T e32 = T(6.0 + std::sqrt(2.0));
  T J[MAXD * MAXD], W[MAXD * MAXD];
  int piv[MAXD];
  jac_u<T>(id, u, p, t, J);
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) W[r * D + c] = (r == c ? T(1) : T(0)) - h * d * J[r * D + c];
  lu_factor<T>(D, W, piv);
  T k1[MAXD], k2[MAXD], k3[MAXD], f1[MAXD], U[MAXD], rhs_v[MAXD] = {};
  lu_solve<T>(D, W, piv, f0, k1);  // k1 = W^{-1} (f0 + h d T), T = 0
  for (int j = 0; j < D; ++j) U[j] = u[j] + (h / 2) * k1[j];
  rhs<T>(id, U, p, t + h / 2, f1);
  for (int j = 0; j < D; ++j) rhs_v[j] = f1[j] - k1[j];
  lu_solve<T>(D, W, piv, rhs_v, k2);
  for (int j = 0; j < D; ++j) k2[j] += k1[j];  // k2 = W^{-1}(f1 - k1) + k1
  for (int j = 0; j < D; ++j) unew[j] = u[j] + h * k2[j];
  rhs<T>(id, unew, p, t + h, f2);
  for (int j = 0; j < D; ++j) rhs_v[j] = f2[j] - e32 * (k2[j] - f1[j]) - 2 * (k1[j] - f0[j]);
  lu_solve<T>(D, W, piv, rhs_v, k3);
  for (int j = 0; j < D; ++j) err[j] = (h / 6) * (k1[j] - 2 * k2[j] + k3[j]);
}

// ----------------------------------------------------------------------------------------------
// Rodas4 and Rodas5P (Sec. 5.2.1: GPURodas4 after Hairer-Wanner, GPURodas5P after Steinebach
// 2023), stiffly accurate Rosenbrock methods of orders 4(3) and 5(4).  They are stepped here in
// the standard form of Hairer-Wanner II, IV.7 for an autonomous f:
//   W = I - h gamma J,   W k_i = h f(y + sum_{j<i} alpha_ij k_j) + h J sum_{j<i} gamma_ij k_j,
//   y_{n+1} = y + sum_j b_j k_j,   yhat = y + sum_j bhat_j k_j,   E = y_{n+1} - yhat.
// The publications give the coefficients for the transformed stages u_i = sum_{j<=i} gamma_ij k_j:
// gamma, a_ij (stage arguments y + sum a_ij u_j) and c_ij (the right-hand sides
// f(...) + sum (c_ij / h) u_j).  With Gamma = (gamma_ij) (gamma on the diagonal) and
// C = (c_ij), Gamma^{-1} = diag(1/gamma) - C and alpha = A Gamma.  Both methods are stiffly
// accurate: the last stage's argument is the embedded solution and y_{n+1} adds u_s, so
// bhat = row s of alpha and b = row s of (alpha + Gamma).
struct RosTab {
  int s = 0;
  double gamma = 0;
  double alpha[8][8] = {}, G[8][8] = {}, b[8] = {}, bhat[8] = {};
};

// transformed coefficients (a, c) -> standard form, as described above
RosTab ros_convert(int s, double gamma, const double (*a)[8], const double (*c)[8]) {
  RosTab t;
  t.s = s;
  t.gamma = gamma;
  // Gamma = (diag(1/gamma) - C)^{-1}: lower triangular, by forward substitution per column
  double Ginv[8][8] = {};
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) Ginv[i][j] = (i == j) ? 1.0 / gamma : (j < i ? -c[i][j] : 0.0);
  for (int col = 0; col < s; ++col)
    for (int i = 0; i < s; ++i) {
      double v = (i == col) ? 1.0 : 0.0;
      for (int j = 0; j < i; ++j) v -= Ginv[i][j] * t.G[j][col];
      t.G[i][col] = v / Ginv[i][i];
    }
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      double v = 0;
      for (int k = 0; k < s; ++k) v += a[i][k] * t.G[k][j];
      t.alpha[i][j] = v;
    }
  for (int j = 0; j < s; ++j) {
    t.bhat[j] = t.alpha[s - 1][j];
    t.b[j] = t.alpha[s - 1][j] + t.G[s - 1][j];
  }
  return t;
}

// Rodas4: Hairer & Wanner, Solving ODEs II (RODAS, 6 stages); stage 6 adds u_5 to stage 5's
// argument (c_5 = c_6 = 1)
RosTab make_rodas4() {
  double a[8][8] = {}, c[8][8] = {};
  a[1][0] = 1.544;
  a[2][0] = 0.9466785280815826; a[2][1] = 0.2557011698983284;
  a[3][0] = 3.314825187068521; a[3][1] = 2.896124015972201; a[3][2] = 0.9986419139977817;
  a[4][0] = 1.221224509226641; a[4][1] = 6.019134481288629; a[4][2] = 12.53708332932087;
  a[4][3] = -0.6878860361058950;
  for (int j = 0; j < 4; ++j) a[5][j] = a[4][j];
  a[5][4] = 1.0;
  c[1][0] = -5.6688;
  c[2][0] = -2.430093356833875; c[2][1] = -0.2063599157091915;
  c[3][0] = -0.1073529058151375; c[3][1] = -9.594562251023355; c[3][2] = -20.47028614809616;
  c[4][0] = 7.496443313967647; c[4][1] = -10.24680431464352; c[4][2] = -33.99990352819905;
  c[4][3] = 11.70890893206160;
  c[5][0] = 8.083246795921522; c[5][1] = -7.981132988064893; c[5][2] = -31.52159432874371;
  c[5][3] = 16.31930543123136; c[5][4] = -6.058818238834054;
  return ros_convert(6, 0.25, a, c);
}

// Rodas5P: Steinebach (2023), 8 stages; stages 7 and 8 each add the previous stage's u to the
// argument before them (c_6 = c_7 = c_8 = 1)
RosTab make_rodas5p() {
  double a[8][8] = {}, c[8][8] = {};
  a[1][0] = 3.0;
  a[2][0] = 2.849394379747939; a[2][1] = 0.45842242204463923;
  a[3][0] = -6.954028509809101; a[3][1] = 2.489845061869568; a[3][2] = -10.358996098473584;
  a[4][0] = 2.8029986275628964; a[4][1] = 0.5072464736228206; a[4][2] = -0.3988312541770524;
  a[4][3] = -0.04721187230404641;
  a[5][0] = -7.502846399306121; a[5][1] = 2.561846144803919; a[5][2] = -11.627539656261098;
  a[5][3] = -0.18268767659942256; a[5][4] = 0.030198172008377946;
  for (int j = 0; j < 5; ++j) a[6][j] = a[5][j];
  a[6][5] = 1.0;
  for (int j = 0; j < 6; ++j) a[7][j] = a[6][j];
  a[7][6] = 1.0;
  c[1][0] = -14.155112264123755;
  c[2][0] = -17.97296035885952; c[2][1] = -2.859693295451294;
  c[3][0] = 147.12150275711716; c[3][1] = -1.41221402718213; c[3][2] = 71.68940251302358;
  c[4][0] = 165.43517024871676; c[4][1] = -0.4592823456491126; c[4][2] = 42.90938336958603;
  c[4][3] = -5.961986721573306;
  c[5][0] = 24.854864614690072; c[5][1] = -3.0009227002832186; c[5][2] = 47.4931110020768;
  c[5][3] = 5.5814197821558125; c[5][4] = -0.6610691825249471;
  c[6][0] = 30.91273214028599; c[6][1] = -3.1208243349937974; c[6][2] = 77.79954646070892;
  c[6][3] = 34.28646028294783; c[6][4] = -19.097331116725623; c[6][5] = -28.087943162872662;
  c[7][0] = 37.80277123390563; c[7][1] = -3.2571969029072276; c[7][2] = 112.26918849496327;
  c[7][3] = 66.9347231244047; c[7][4] = -40.06618937091002; c[7][5] = -54.66780262877968;
  c[7][6] = -9.48861652309627;
  return ros_convert(8, 0.21193756319429014, a, c);
}

const RosTab& ros_tab(int alg) {
  static const RosTab r4 = make_rodas4(), r5 = make_rodas5p();
  return alg == ALG_RODAS4 ? r4 : r5;
}

// One Rodas4 / Rodas5P step from u with f0 = f(u) (the first stage's f).  Fills unew = y_{n+1},
// err = E and f1 = f(unew) (the next step's f0).
template <class T>
void rodas_step(int alg, int id, int D, const T* u, const T* p, T t, T h, const T* f0, T* unew,
                T* err, T* f1) {
  const RosTab& tb = ros_tab(alg);
  const int s = tb.s;
  T J[MAXD * MAXD], W[MAXD * MAXD];
  int piv[MAXD];
  jac_u<T>(id, u, p, t, J);
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c)
      W[r * D + c] = (r == c ? T(1) : T(0)) - h * T(tb.gamma) * J[r * D + c];
  lu_factor<T>(D, W, piv);
  T k[8][MAXD];
  for (int i = 0; i < s; ++i) {
    T g[MAXD], fi[MAXD], v[MAXD], r[MAXD];
    for (int j = 0; j < D; ++j) {
      g[j] = u[j];
      v[j] = T(0);
      for (int l = 0; l < i; ++l) {
        g[j] += T(tb.alpha[i][l]) * k[l][j];
        v[j] += T(tb.G[i][l]) * k[l][j];
      }
    }
    if (i == 0) {
      for (int j = 0; j < D; ++j) fi[j] = f0[j];
    } else {
      rhs<T>(id, g, p, t, fi);  // autonomous models: the stage time does not enter f
    }
    for (int row = 0; row < D; ++row) {
      T Jv = T(0);
      for (int c = 0; c < D; ++c) Jv += J[row * D + c] * v[c];
      r[row] = h * fi[row] + h * Jv;
    }
    lu_solve<T>(D, W, piv, r, k[i]);
  }
  for (int j = 0; j < D; ++j) {
    T y1 = u[j], yh = u[j];
    for (int l = 0; l < s; ++l) {
      y1 += T(tb.b[l]) * k[l][j];
      yh += T(tb.bhat[l]) * k[l][j];
    }
    unew[j] = y1;
    err[j] = y1 - yh;
  }
  rhs<T>(id, unew, p, t + h, f1);
}

bool is_rosenbrock(int alg) { return alg == ALG_ROS23 || alg == ALG_RODAS4 || alg == ALG_RODAS5P; }

// ----------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 Philox S-box with a Weyl key
// schedule.  Round: (c0,c1,c2,c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)).
void philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = uint64_t(M0) * uint64_t(c[0]);
    uint64_t p1 = uint64_t(M1) * uint64_t(c[2]);
    uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
    uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
    uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Standard normal number `k` of trajectory stream `traj` (fp64: 2 normals per Philox call,
// fp32: 4 normals per call).  Computed in double from exact uniforms.
double normal_draw(uint64_t seed, uint64_t traj, uint64_t k, bool fp64) {
  const double PI = 3.14159265358979323846;
  uint64_t call = fp64 ? (k >> 1) : (k >> 2);
  uint32_t ctr[4] = {uint32_t(call), uint32_t(call >> 32), uint32_t(traj), uint32_t(traj >> 32)};
  uint32_t key[2] = {uint32_t(seed), uint32_t(seed >> 32)};
  uint32_t x[4];
  philox(ctr, key, x);
  double ua, ub;
  int which;
  if (fp64) {
    uint64_t a = (uint64_t(x[0]) << 32) | x[1];
    uint64_t b = (uint64_t(x[2]) << 32) | x[3];
    ua = (double(a >> 12) + 0.5) * std::ldexp(1.0, -52);
    ub = (double(b >> 12) + 0.5) * std::ldexp(1.0, -52);
    which = int(k & 1);
  } else {
    int pair = int((k & 3) >> 1);
    ua = (double(x[2 * pair] >> 9) + 0.5) * std::ldexp(1.0, -23);
    ub = (double(x[2 * pair + 1] >> 9) + 0.5) * std::ldexp(1.0, -23);
    which = int(k & 1);
  }
  double r = std::sqrt(-2.0 * std::log(ua));
  return which == 0 ? r * std::cos(2.0 * PI * ub) : r * std::sin(2.0 * PI * ub);
}

// ----------------------------------------------------------------------------------------------
struct Opts {
  int rhs, alg, D, P, Mw;
  double dt, abstol, reltol, dt0;
  long long maxiters;
  const double* saveat;
  int n_save;
  unsigned long long seed;
  long long index_offset;
  bool stream_fp64;  // normals from the FP64 stream (2 per Philox call) or the FP32 one (4)
  bool dense;        // adaptive Tsit5: save times by the dense output, steps not cut at them
  double dtmax;      // adaptive methods: largest step (<= 0: none)
};

// Hairer-Norsett-Wanner I, II.4: starting step size for an order-p method.
template <class T>
T initial_step(const Opts& o, const T* u0, const T* p, T t0, const T* f0, int order,
               long long* fevals) {
  const int D = o.D;
  T sc[MAXD], tmp[MAXD], u1[MAXD], f1[MAXD];
  for (int j = 0; j < D; ++j) sc[j] = T(o.abstol) + T(o.reltol) * std::fabs(u0[j]);
  T d0 = rms_scaled(u0, sc, D);
  T d1 = rms_scaled(f0, sc, D);
  T h0 = (d0 < T(1e-5) || d1 < T(1e-5)) ? T(1e-6) : T(0.01) * d0 / d1;
  for (int j = 0; j < D; ++j) u1[j] = u0[j] + h0 * f0[j];
  rhs<T>(o.rhs, u1, p, t0 + h0, f1);
  *fevals += 1;
  for (int j = 0; j < D; ++j) tmp[j] = f1[j] - f0[j];
  T d2 = rms_scaled(tmp, sc, D) / h0;
  T dm = std::max(d1, d2);
  T h1 = (dm <= T(1e-15)) ? std::max(T(1e-6), h0 * T(1e-3))
                          : std::pow(T(0.01) / dm, T(1.0 / (order + 1)));
  return std::min(T(100) * h0, h1);
}

template <class T>
struct Traj {
  const Opts* o;
  T u[MAXD], p[MAXP];
  T t0, tf;
  T* out;  // [S or 1][D] row-major scratch owned by the caller
  int S;
  signed char status;
  long long accepted, rejected, fevals, events;
  // every-step record (adaptive methods): entry k = (t, u) after k accepted steps, k < cap
  T* rec_t = nullptr;
  T* rec_u = nullptr;
  int cap = 0;
  void record(T t) {
    if (accepted < cap) {
      rec_t[accepted] = t;
      for (int j = 0; j < o->D; ++j) rec_u[accepted * o->D + j] = u[j];
    }
  }
};

template <class T>
void fill_nan(T* v, int n) {
  for (int i = 0; i < n; ++i) v[i] = std::numeric_limits<T>::quiet_NaN();
}

// ---- the weak order 2 stochastic Runge-Kutta step (GPUSIEA, Sec. 5.2.2) ------------------------
// The paper names a weak second-order method of Tocino and Vigo-Aguiar for diagonal noise and
// writes the explicit stochastic Runge-Kutta family it belongs to (Sec. 3.3: stage values
// eta_j, weights alpha_j for the drift and beta_j for the noise, and a fit term R), but prints
// no scheme.  Taken: the weak second-order scheme of improved-Euler type in that family
// (Kloeden and Platen, the explicit weak order 2.0 scheme), per component j with its own
// increment dW_j and diffusion b_j depending on component j:
//   Ybar = X + a(X) h + b(X) dW,     Y+- = X + a(X) h +- b(X) sqrt(h),
//   X_{n+1} = X + (a(X) + a(Ybar)) h / 2 + (b(Y+) + b(Y-) + 2 b(X)) dW / 4
//                 + (b(Y+) - b(Y-)) (dW^2 - h) / (4 sqrt(h)),
// the last term being the fit term R.  With b = 0 it is Heun's (improved Euler) method.
template <class T>
void siea_step(int id, int D, int Mw, const T* u, const T* p, T t, T h, const T* z, T* unew) {
  T a0[MAXD], a1[MAXD], G[MAXD * 8], b0[MAXD], bp[MAXD], bm[MAXD], Y[MAXD], dW[MAXD];
  const T sq = std::sqrt(h);
  rhs<T>(id, u, p, t, a0);
  diffusion<T>(id, u, p, t, G);
  for (int j = 0; j < D; ++j) {
    b0[j] = G[j * Mw + j];
    dW[j] = sq * z[j];
  }
  for (int j = 0; j < D; ++j) Y[j] = u[j] + a0[j] * h + b0[j] * dW[j];  // Ybar
  rhs<T>(id, Y, p, t + h, a1);
  for (int j = 0; j < D; ++j) Y[j] = u[j] + a0[j] * h + b0[j] * sq;     // Y+
  diffusion<T>(id, Y, p, t + h, G);
  for (int j = 0; j < D; ++j) bp[j] = G[j * Mw + j];
  for (int j = 0; j < D; ++j) Y[j] = u[j] + a0[j] * h - b0[j] * sq;     // Y-
  diffusion<T>(id, Y, p, t + h, G);
  for (int j = 0; j < D; ++j) bm[j] = G[j * Mw + j];
  for (int j = 0; j < D; ++j)
    unew[j] = u[j] + (a0[j] + a1[j]) * h / T(2) + (bp[j] + bm[j] + T(2) * b0[j]) * dW[j] / T(4) +
              (bp[j] - bm[j]) * (dW[j] * dW[j] - h) / (T(4) * sq);
}

// ---- fixed-step drivers (Tsit5 fixed, RK4, Euler-Maruyama, SIEA) -------------------------------
// n = ceil((tf - t0)/dt - 1e-12); steps 0..n-2 use h = dt, the last uses tf - (t0 + (n-1) dt);
// step k starts at t_k = t0 + k dt.  A save time s is recorded after step
// k_s = ceil((s - t0)/dt - 1e-12) (clamped to [0, n]); save times outside [t0, tf] give NaN.
template <class T>
void solve_fixed(Traj<T>& tr, uint64_t traj_index) {
  const Opts& o = *tr.o;
  const int D = o.D;
  const double t0 = double(tr.t0), tf = double(tr.tf), dt = o.dt;
  long long n = (tf > t0) ? (long long)std::ceil((tf - t0) / dt - 1e-12) : 0;
  if (n < 0) n = 0;
  long long nrun = std::min(n, o.maxiters);
  const T h_reg = T(dt);
  const T h_last = n > 0 ? T(tf - (t0 + double(n - 1) * dt)) : T(0);
  const int S = o.n_save;  // number of save times (0: final state only)
  const bool save_mode = o.n_save > 0;
  auto ks_of = [&](int si) -> long long {
    double s = o.saveat[si];
    if (s < t0 || s > tf) return -1;
    long long ks = (s <= t0) ? 0 : (long long)std::ceil((s - t0) / dt - 1e-12);
    return std::min(std::max(ks, 0LL), n);
  };
  if (save_mode) fill_nan(tr.out, S * D);
  int si = 0;
  auto record_saves = [&](long long step_count) {
    while (si < S) {
      long long ks = ks_of(si);
      if (ks < 0) { ++si; continue; }
      if (ks != step_count) break;
      for (int j = 0; j < D; ++j) tr.out[si * D + j] = tr.u[j];
      ++si;
    }
  };
  if (save_mode) record_saves(0);
  T k1[MAXD];
  if (o.alg == ALG_TSIT5_FIXED) {
    rhs<T>(o.rhs, tr.u, tr.p, tr.t0, k1);
    tr.fevals += 1;
  }
  for (long long k = 0; k < nrun; ++k) {
    const T h = (k == n - 1) ? h_last : h_reg;
    const T tk = T(t0) + T(k) * T(dt);
    T unew[MAXD];
    if (o.alg == ALG_TSIT5_FIXED) {
      T err[MAXD], k7[MAXD];
      tsit5_step<T>(o.rhs, D, tr.u, tr.p, tk, h, k1, unew, err, k7);
      for (int j = 0; j < D; ++j) k1[j] = k7[j];
      tr.fevals += 6;
    } else if (o.alg == ALG_RK4) {
      rk4_step<T>(o.rhs, D, tr.u, tr.p, tk, h, unew);
      tr.fevals += 4;
    } else if (o.alg == ALG_SIEA) {
      // weak order 2 (Sec. 5.2.2, GPUSIEA), diagonal noise: step k uses normal k*Mw + j
      // for component j, dW_j = sqrt(h) Z_{k,j}
      T z[MAXD];
      for (int j = 0; j < D; ++j)
        z[j] = T(normal_draw(o.seed, traj_index, uint64_t(k) * uint64_t(o.Mw) + uint64_t(j),
                             o.stream_fp64));
      siea_step<T>(o.rhs, D, o.Mw, tr.u, tr.p, tk, h, z, unew);
      tr.fevals += 2;
    } else {  // Euler-Maruyama (Sec. 3.3): X_{k+1} = X_k + a(X_k) h + sum_m b_m(X_k) dW_m,
      // dW_m = sqrt(h) Z_{k,m}; Z_{k,m} is normal number k*Mw + m of the trajectory's stream
      const int Mw = o.Mw;
      T a[MAXD], G[MAXD * 8], z[MAXD];
      rhs<T>(o.rhs, tr.u, tr.p, tk, a);
      diffusion<T>(o.rhs, tr.u, tr.p, tk, G);
      tr.fevals += 1;
      for (int m = 0; m < Mw; ++m)
        z[m] = T(normal_draw(o.seed, traj_index, uint64_t(k) * uint64_t(Mw) + uint64_t(m),
                             o.stream_fp64));
      T sq = std::sqrt(h);
      for (int j = 0; j < D; ++j) {
        T x = tr.u[j] + a[j] * h;
        for (int m = 0; m < Mw; ++m) x = x + G[j * Mw + m] * sq * z[m];
        unew[j] = x;
      }
    }
    for (int j = 0; j < D; ++j) tr.u[j] = unew[j];
    tr.accepted += 1;
    if (save_mode) record_saves(k + 1);
  }
  if (nrun < n) tr.status = ST_MAXITERS;
  else if (!finite_all(tr.u, D)) tr.status = ST_NONFINITE;
  if (!save_mode)
    for (int j = 0; j < D; ++j) tr.out[j] = tr.u[j];
}

// ---- adaptive drivers (Tsit5 with PI control, Rosenbrock23) -----------------------------------
template <class T>
void solve_adaptive(Traj<T>& tr) {
  const Opts& o = *tr.o;
  const int D = o.D;
  // Rosenbrock methods (no dense output, no events); the controller's exponent denominator k
  // is the error estimate's order + 1: Tsit5 5(4) and Rodas5P 5(4): 5, Rodas4 4(3): 4,
  // Rosenbrock23 2(3): 3; the starting step uses the order of the advancing solution
  const bool is_ros = is_rosenbrock(o.alg);
  const int k_ord = o.alg == ALG_ROS23 ? 3 : o.alg == ALG_RODAS4 ? 4 : 5;
  const int p_ord = o.alg == ALG_ROS23 ? 2 : o.alg == ALG_RODAS4 ? 4 : 5;
  const T beta1 = T(0.7 / k_ord), beta2 = T(0.4 / k_ord), rej_exp = T(1.0 / k_ord);
  const T atol = T(o.abstol), rtol = T(o.reltol);
  const int S = o.n_save;  // number of save times (0: final state only)
  const bool save_mode = o.n_save > 0;
  if (save_mode) fill_nan(tr.out, S * D);

  Clock<T> clk;
  clk.set(tr.t0);
  int si = 0;
  // skip save times before t0
  while (si < S && T(o.saveat[si]) < tr.t0) ++si;

  T fcur[MAXD];  // k1 (Tsit5) or f0 (R23): f at the current state
  rhs<T>(o.rhs, tr.u, tr.p, tr.t0, fcur);
  tr.fevals += 1;
  T h;
  if (o.dt0 > 0) h = T(o.dt0);
  else h = initial_step<T>(o, tr.u, tr.p, tr.t0, fcur, p_ord, &tr.fevals);
  T qold = T(QOLD_INIT);
  long long attempts = 0;
  const bool dense = o.dense && !is_ros && save_mode;
  const bool ev = has_event(o.rhs) && !is_ros;
  long long events = 0;
  if (tr.rec_t) tr.record(tr.t0);  // entry 0: the initial state
  if (dense)  // save times equal to t0 take u0; the steps then run to tf uncut
    while (si < S && T(o.saveat[si]) == tr.t0 && tr.t0 <= tr.tf) {
      for (int j = 0; j < D; ++j) tr.out[si * D + j] = tr.u[j];
      ++si;
    }

  for (;;) {
    const bool stop_is_save = !dense && (si < S && T(o.saveat[si]) < tr.tf);
    const T stop = stop_is_save ? T(o.saveat[si]) : tr.tf;
    const T rem = clk.remaining(stop);
    if (rem <= T(STOP_EPS) * std::max(T(1), std::fabs(stop))) {
      clk.set(stop);
      if (stop_is_save) {
        for (int j = 0; j < D; ++j) tr.out[si * D + j] = tr.u[j];
        ++si;
        continue;
      }
      // reached tf: record every remaining save time equal to tf (dense: any save left
      // within the last STOP_EPS of the span)
      while (si < S && (T(o.saveat[si]) == tr.tf || (dense && T(o.saveat[si]) <= tr.tf))) {
        for (int j = 0; j < D; ++j) tr.out[si * D + j] = tr.u[j];
        ++si;
      }
      break;
    }
    if (attempts >= o.maxiters) { tr.status = ST_MAXITERS; break; }
    const T hcap = (o.dtmax > 0) ? std::min(h, T(o.dtmax)) : h;
    const bool last = (hcap >= rem);
    const T hs = last ? rem : hcap;
    const T tnow = clk.value();
    if (hs < T(Prec<T>::dtmin_factor) * std::max(T(1), std::fabs(tnow))) {
      tr.status = ST_DT_MIN;
      break;
    }
    T unew[MAXD], err[MAXD], fnew[MAXD], kst[7][MAXD];
    if (o.alg == ALG_ROS23) {
      ros23_step<T>(o.rhs, D, tr.u, tr.p, tnow, hs, fcur, unew, err, fnew);
      tr.fevals += 2;
    } else if (is_ros) {  // Rodas4 / Rodas5P: stages 2..s and f(u_{n+1})
      rodas_step<T>(o.alg, o.rhs, D, tr.u, tr.p, tnow, hs, fcur, unew, err, fnew);
      tr.fevals += ros_tab(o.alg).s;
    } else {
      tsit5_step<T>(o.rhs, D, tr.u, tr.p, tnow, hs, fcur, unew, err, fnew,
                    (dense || ev) ? kst : nullptr);
      tr.fevals += 6;
    }
    ++attempts;
    // q = || E / (atol + rtol max(|u(t)|, |u(t+h)|)) ||  (RMS norm)
    T sc[MAXD];
    for (int j = 0; j < D; ++j)
      sc[j] = atol + rtol * std::max(std::fabs(tr.u[j]), std::fabs(unew[j]));
    const T q = rms_scaled(err, sc, D);
    // NONFINITE: u_{n+1} has a NaN/Inf component or q is NaN; q = +Inf is an ordinary reject.
    if (std::isnan(q) || !finite_all(unew, D)) { tr.status = ST_NONFINITE; break; }
    if (q <= T(1)) {
      const T qg = std::max(q, T(Q_FLOOR));
      T fac = T(ETA) * std::pow(qg, -beta1) * std::pow(qold, beta2);
      fac = std::min(T(FAC_MAX), std::max(T(FAC_MIN), fac));
      qold = std::max(q, T(QOLD_INIT));
      T th_ev = -1, cq[4][MAXD];
      if (ev) {
        dense_coeffs<T>(D, hs, kst, cq);
        th_ev = find_event<T>(o.rhs, D, tr.u, unew, tr.p, tnow, hs, cq);
      }
      const bool cut = th_ev > 0 && th_ev < 1;  // the step ends at the event
      if (dense) {  // save times in (t_n, t_n + hs] (up to the event): theta = (s - t_n) / hs
        while (si < S) {
          const T sv = T(o.saveat[si]);
          if (sv > tr.tf) break;
          const T rs = clk.remaining(sv);
          const bool at_end = !cut && last && sv == stop;
          if (!at_end && rs > (cut ? th_ev * hs : hs)) break;
          if (at_end)
            for (int j = 0; j < D; ++j) tr.out[si * D + j] = unew[j];
          else
            tsit5_dense<T>(D, tr.u, hs, kst, rs / hs, tr.out + si * D);
          ++si;
        }
      }
      if (th_ev > 0) {  // state at the event, then the affect; f is evaluated afresh
        if (cut) dense_poly<T>(D, tr.u, cq, th_ev, unew);
        event_affect<T>(o.rhs, unew, tr.p, tnow + th_ev * hs);
        rhs<T>(o.rhs, unew, tr.p, tnow + th_ev * hs, fnew);
        tr.fevals += 1;
        ++events;
      }
      for (int j = 0; j < D; ++j) { tr.u[j] = unew[j]; fcur[j] = fnew[j]; }
      tr.events = events;
      if (cut) clk.add(th_ev * hs);
      else if (last) clk.set(stop);
      else clk.add(hs);
      tr.accepted += 1;
      if (tr.rec_t) tr.record(clk.value());
      h = hs * fac;
    } else {
      const T qg = std::max(q, T(Q_FLOOR));
      const T fac = std::max(T(FAC_MIN), T(ETA) * std::pow(qg, -rej_exp));
      tr.rejected += 1;
      h = hs * fac;
    }
  }
  if (!save_mode)
    for (int j = 0; j < D; ++j) tr.out[j] = tr.u[j];
}

// index helpers for the two supported layouts
inline long long idx_in(int layout, long long i, int k, long long N, int width) {
  return layout == LAYOUT_SOA ? (long long)k * N + i : i * width + k;
}
inline long long idx_out(int layout, long long i, int s, int k, long long N, int S, int D) {
  return layout == LAYOUT_SOA ? ((long long)s * D + k) * N + i : (i * S + s) * (long long)D + k;
}

template <class T>
void solve_range(const Opts& o, int layout, long long N, long long i0, long long i1,
                 const double* params, const double* u0, const double* tspan, double* out,
                 signed char* status, long long* stats, long long* events,
                 int cap = 0, double* rec_t = nullptr, double* rec_u = nullptr,
                 long long* rec_n = nullptr) {
  const int D = o.D, P = o.P;
  const int S = o.n_save > 0 ? o.n_save : 1;
  std::vector<T> buf(size_t(S) * D), rt(static_cast<size_t>(cap)), ru(static_cast<size_t>(cap) * D);
  for (long long i = i0; i < i1; ++i) {
    Traj<T> tr;
    tr.o = &o;
    for (int k = 0; k < P; ++k) tr.p[k] = T(params[idx_in(layout, i, k, N, P)]);
    for (int k = 0; k < D; ++k) tr.u[k] = T(u0[idx_in(layout, i, k, N, D)]);
    tr.t0 = T(tspan[idx_in(layout, i, 0, N, 2)]);
    tr.tf = T(tspan[idx_in(layout, i, 1, N, 2)]);
    tr.out = buf.data();
    tr.S = S;
    tr.status = ST_OK;
    tr.accepted = tr.rejected = tr.fevals = tr.events = 0;
    if (cap > 0) {
      tr.cap = cap;
      tr.rec_t = rt.data();
      tr.rec_u = ru.data();
    }
    if (o.alg == ALG_TSIT5_ADAPTIVE || is_rosenbrock(o.alg)) solve_adaptive<T>(tr);
    else solve_fixed<T>(tr, uint64_t(o.index_offset + i));
    if (cap > 0) {  // row-major [N][cap] / [N][cap][D]; unused entries NaN
      const long long n = std::min<long long>(tr.accepted + 1, cap);
      for (int k = 0; k < cap; ++k) {
        rec_t[i * cap + k] = k < n ? double(rt[k]) : std::numeric_limits<double>::quiet_NaN();
        for (int j = 0; j < D; ++j)
          rec_u[(i * cap + k) * D + j] =
              k < n ? double(ru[k * D + j]) : std::numeric_limits<double>::quiet_NaN();
      }
      rec_n[i] = tr.accepted + 1;
    }
    for (int s = 0; s < S; ++s)
      for (int k = 0; k < D; ++k) out[idx_out(layout, i, s, k, N, S, D)] = double(buf[s * D + k]);
    if (status) status[i] = tr.status;
    if (stats) {
      stats[i * 3 + 0] = tr.accepted;
      stats[i * 3 + 1] = tr.rejected;
      stats[i * 3 + 2] = tr.fevals;
    }
    if (events) events[i] = tr.events;
  }
}

template <class F>
void parallel_for(long long N, int nthreads, F&& fn) {
  if (nthreads <= 1 || N < 2) {
    fn(0LL, N);
    return;
  }
  std::vector<std::thread> th;
  // interleaved chunks of 64 so that slow and fast trajectories spread over the threads
  const long long chunk = 64;
  const long long nchunks = (N + chunk - 1) / chunk;
  for (int w = 0; w < nthreads; ++w) {
    th.emplace_back([&, w]() {
      for (long long c = w; c < nchunks; c += nthreads) {
        long long a = c * chunk, b = std::min(N, a + chunk);
        fn(a, b);
      }
    });
  }
  for (auto& t : th) t.join();
}

}  // namespace

// ================================================================================================
extern "C" {

// Solve N trajectories.  All arrays are host double arrays; `layout` 0 = row-major
// (params[N][P], u0[N][D], tspan[N][2], out[N][S][D]), 1 = structure of arrays
// (params[P][N], u0[D][N], tspan[2][N], out[S][D][N]).  `precision` 0 = FP64, 1 = FP32 mode
// (inputs rounded to float first by the caller; arithmetic in float, time compensated),
// 2 = FP64 arithmetic driven by the FP32 normal stream (the reference for FP32 SDE paths).
// stats[N][3] = accepted, rejected, f-evaluations; events[N] (or NULL) = events handled.
// dense: adaptive Tsit5 saves by the dense output; dtmax > 0 caps adaptive steps.
// Returns 0, or -1 on bad arguments.
int oracle_solve(int rhs_id, int alg, int precision, int layout, long long N,
                 const double* params, const double* u0, const double* tspan, double dt,
                 double abstol, double reltol, double dt0, long long maxiters,
                 const double* saveat, int n_save, unsigned long long seed,
                 long long index_offset, double* out, signed char* status, long long* stats,
                 int nthreads, int dense, double dtmax, long long* events) {
  Model m = model_of(rhs_id);
  if (m.D == 0 || N < 0 || alg < 1 || alg > 8) return -1;
  if (alg == ALG_EM && m.Mw == 0) return -1;  // Euler-Maruyama needs an SDE model
  if (alg == ALG_SIEA && (m.Mw == 0 || m.Mw != m.D)) return -1;  // diagonal noise only
  if (rhs_id == RHS_CRN && alg != ALG_EM) return -1;
  if (is_rosenbrock(alg) && rhs_id == RHS_BALL) return -1;  // no Jacobian
  if (alg == ALG_SIEA && rhs_id != RHS_GBM) return -1;
  if (has_event(rhs_id) && alg != ALG_TSIT5_ADAPTIVE) return -1;  // events need the interpolant
  if (precision < 0 || precision > 2) return -1;
  Opts o{rhs_id, alg, m.D, m.P, m.Mw, dt, abstol, reltol, dt0, maxiters, saveat, n_save, seed,
         index_offset, precision == 0, dense != 0, dtmax};
  parallel_for(N, nthreads, [&](long long a, long long b) {
    if (precision != 1)
      solve_range<double>(o, layout, N, a, b, params, u0, tspan, out, status, stats, events);
    else
      solve_range<float>(o, layout, N, a, b, params, u0, tspan, out, status, stats, events);
  });
  return 0;
}

// Every accepted step of adaptive solves (Tsit5, Rosenbrock23): rec_t[N][cap], rec_u[N][cap][D]
// (row-major) hold (t, u) after k = 0, 1, ... accepted steps (k = 0: the initial state), the
// entries past the count NaN; rec_n[N] = accepted steps + 1, which may exceed cap (the
// record then holds the first cap).  out / status / stats as for oracle_solve (final state).
int oracle_solve_steps(int rhs_id, int alg, int precision, long long N, const double* params,
                       const double* u0, const double* tspan, double abstol, double reltol,
                       double dt0, long long maxiters, double dtmax, int cap, double* out,
                       signed char* status, long long* stats, double* rec_t, double* rec_u,
                       long long* rec_n, int nthreads) {
  Model m = model_of(rhs_id);
  if (m.D == 0 || N < 0 || cap < 1) return -1;
  if (alg != ALG_TSIT5_ADAPTIVE && !is_rosenbrock(alg)) return -1;
  if (rhs_id == RHS_CRN || (has_event(rhs_id) && alg != ALG_TSIT5_ADAPTIVE)) return -1;
  if (precision < 0 || precision > 1) return -1;
  Opts o{rhs_id, alg, m.D, m.P, m.Mw, 0.0, abstol, reltol, dt0, maxiters, nullptr, 0, 0, 0,
         precision == 0, false, dtmax};
  parallel_for(N, nthreads, [&](long long a, long long b) {
    if (precision == 0)
      solve_range<double>(o, 0, N, a, b, params, u0, tspan, out, status, stats, nullptr, cap,
                          rec_t, rec_u, rec_n);
    else
      solve_range<float>(o, 0, N, a, b, params, u0, tspan, out, status, stats, nullptr, cap,
                         rec_t, rec_u, rec_n);
  });
  return 0;
}

// One step of a method (for convergence-order and stability pins).  alg: 1 Tsit5, 3 RK4,
// 4 Rosenbrock23, 5 Euler-Maruyama and 8 SIEA with the given normal z (GBM), 6 Rodas4,
// 7 Rodas5P.  err (Tsit5, Rosenbrock methods) may be NULL.
int oracle_step(int rhs_id, int alg, const double* u, const double* p, double t, double h,
                double z, double* unew, double* err) {
  Model m = model_of(rhs_id);
  if (m.D == 0) return -1;
  if (is_rosenbrock(alg) && (rhs_id == RHS_CRN || rhs_id == RHS_BALL)) return -1;  // no Jacobian
  double e[MAXD] = {0}, fx[MAXD], k1[MAXD];
  if (alg == ALG_TSIT5_FIXED || alg == ALG_TSIT5_ADAPTIVE) {
    rhs<double>(rhs_id, u, p, t, k1);
    tsit5_step<double>(rhs_id, m.D, u, p, t, h, k1, unew, e, fx);
  } else if (alg == ALG_RK4) {
    rk4_step<double>(rhs_id, m.D, u, p, t, h, unew);
  } else if (alg == ALG_ROS23) {
    rhs<double>(rhs_id, u, p, t, k1);
    ros23_step<double>(rhs_id, m.D, u, p, t, h, k1, unew, e, fx);
  } else if (alg == ALG_RODAS4 || alg == ALG_RODAS5P) {
    rhs<double>(rhs_id, u, p, t, k1);
    rodas_step<double>(alg, rhs_id, m.D, u, p, t, h, k1, unew, e, fx);
  } else if (alg == ALG_SIEA) {
    if (rhs_id != RHS_GBM) return -1;
    const double zz[1] = {z};
    siea_step<double>(rhs_id, m.D, m.Mw, u, p, t, h, zz, unew);
  } else if (alg == ALG_EM) {
    if (rhs_id != RHS_GBM) return -1;
    double a[MAXD], b[MAXD];
    f_gbm<double>(u, p, t, a);
    g_gbm<double>(u, p, t, b);
    for (int j = 0; j < m.D; ++j) unew[j] = u[j] + a[j] * h + b[j] * std::sqrt(h) * z;
  } else {
    return -1;
  }
  if (err)
    for (int j = 0; j < m.D; ++j) err[j] = e[j];
  return 0;
}

void oracle_pollu_reaction_sum(const double* y, const double* k, double* dy) {
  pollu_reaction_sum(y, k, dy);
}

void oracle_tsit5_dense(double* r) {
  for (int i = 0; i < 7; ++i)
    for (int q = 0; q < 4; ++q) r[i * 4 + q] = TS_DENSE[i][q];
}

// The standard-form coefficients the oracle steps Rodas4 (alg 6) / Rodas5P (alg 7) with:
// returns s and fills gamma, alpha[s][s], Gamma[s][s] (gamma on the diagonal), b[s], bhat[s]
// (arrays of 8 x 8 / 8 entries, row-major with stride 8); -1 for another alg.
int oracle_rosenbrock_tableau(int alg, double* gamma, double* alpha, double* G, double* b,
                              double* bhat) {
  if (alg != ALG_RODAS4 && alg != ALG_RODAS5P) return -1;
  const RosTab& t = ros_tab(alg);
  *gamma = t.gamma;
  for (int i = 0; i < 8; ++i) {
    b[i] = t.b[i];
    bhat[i] = t.bhat[i];
    for (int j = 0; j < 8; ++j) {
      alpha[i * 8 + j] = t.alpha[i][j];
      G[i * 8 + j] = t.G[i][j];
    }
  }
  return t.s;
}

void oracle_tsit5_tableau(double* c, double* A, double* b, double* bhat) {
  for (int i = 0; i < 7; ++i) {
    c[i] = TS_C[i];
    b[i] = TS_B[i];
    bhat[i] = TS_BHAT[i];
    for (int j = 0; j < 7; ++j) A[i * 7 + j] = TS_A[i][j];
  }
}

int oracle_rhs(int rhs_id, const double* u, const double* p, double t, double* du) {
  if (model_of(rhs_id).D == 0) return -1;
  rhs<double>(rhs_id, u, p, t, du);
  return 0;
}

// Diffusion matrix G[D][Mw] of an SDE model (GBM, CRN).
int oracle_diffusion(int rhs_id, const double* u, const double* p, double t, double* G) {
  if (model_of(rhs_id).Mw == 0) return -1;
  diffusion<double>(rhs_id, u, p, t, G);
  return 0;
}

// One Euler-Maruyama step with the given normals z[Mw] (any SDE model).
int oracle_em_step(int rhs_id, const double* u, const double* p, double t, double h,
                   const double* z, double* unew) {
  const Model m = model_of(rhs_id);
  if (m.Mw == 0) return -1;
  double a[MAXD], G[MAXD * 8];
  rhs<double>(rhs_id, u, p, t, a);
  diffusion<double>(rhs_id, u, p, t, G);
  const double sq = std::sqrt(h);
  for (int j = 0; j < m.D; ++j) {
    double x = u[j] + a[j] * h;
    for (int k = 0; k < m.Mw; ++k) x = x + G[j * m.Mw + k] * sq * z[k];
    unew[j] = x;
  }
  return 0;
}

int oracle_jac(int rhs_id, const double* u, const double* p, double t, double* Ju, double* Jp) {
  if (model_of(rhs_id).D == 0 || rhs_id == RHS_CRN || rhs_id == RHS_BALL) return -1;
  if (Jp && rhs_id >= RHS_OREGO) return -1;  // no df/dp for the stiff test models
  if (Ju) jac_u<double>(rhs_id, u, p, t, Ju);
  if (Jp) jac_p<double>(rhs_id, u, p, t, Jp);
  return 0;
}

// Solve W x = b by the oracle's LU (for the linear-algebra pin).
int oracle_lu_solve(int D, const double* W, const double* b, double* x) {
  if (D < 1 || D > MAXD) return -1;
  double LU[MAXD * MAXD];
  int piv[MAXD];
  std::memcpy(LU, W, sizeof(double) * D * D);
  lu_factor<double>(D, LU, piv);
  lu_solve<double>(D, LU, piv, b, x);
  return 0;
}

void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox(ctr, key, out);
}

// normals z_0..z_{n-1} of the stream of trajectory `traj`
void oracle_normals(unsigned long long seed, unsigned long long traj, long long n, int fp64,
                    double* out) {
  for (long long k = 0; k < n; ++k) out[k] = normal_draw(seed, traj, uint64_t(k), fp64 != 0);
}

// Classic RK4 as an explicit tableau (used by the tangent gradient below; the forward solver
// above steps RK4 with the textbook formula).
const double RK4_C[4] = {0.0, 0.5, 0.5, 1.0};
const double RK4_A[4][4] = {{0, 0, 0, 0}, {0.5, 0, 0, 0}, {0, 0.5, 0, 0}, {0, 0, 1.0, 0}};
const double RK4_B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

// Exact gradient of a discrete fixed-step explicit Runge-Kutta map (FP64) by forward-mode
// tangents: alg 1 = Tsit5 (7-stage tableau, b_7 = 0), alg 3 = RK4.
// For each trajectory i: g_p[i][m] = sum_k grad_out[i][k] d u_k(tf) / d p_m,
// g_u0[i][j] = sum_k grad_out[i][k] d u_k(tf) / d u0_j.  Row-major arrays.
// Tangent recursion (chain rule through every stage, Sec. 3.1 stage equations):
// dU_i = du + h sum_j a_ij dk_j,  dk_i = f_u(U_i) dU_i + f_p(U_i) dtheta,
// du_{n+1} = du_n + h sum_i b_i dk_i.
int oracle_fixed_grad(int rhs_id, int alg_id, long long N, const double* params,
                      const double* u0, const double* tspan, double dt, const double* grad_out,
                      double* g_p, double* g_u0, double* u_final, int nthreads) {
  int S = 0;
  const double* TC = nullptr;
  const double* TB = nullptr;
  double TA[7][7] = {};
  if (alg_id == ALG_TSIT5_FIXED) {
    S = 7;
    TC = TS_C;
    TB = TS_B;
    for (int r = 0; r < 7; ++r)
      for (int q = 0; q < 7; ++q) TA[r][q] = TS_A[r][q];
  } else if (alg_id == ALG_RK4) {
    S = 4;
    TC = RK4_C;
    TB = RK4_B;
    for (int r = 0; r < 4; ++r)
      for (int q = 0; q < 4; ++q) TA[r][q] = RK4_A[r][q];
  } else {
    return -1;
  }
  Model m = model_of(rhs_id);
  if (m.D == 0 || rhs_id == RHS_CRN || rhs_id >= RHS_BALL) return -1;  // needs df/du, df/dp
  const int D = m.D, P = m.P, M = m.P + m.D;
  parallel_for(N, nthreads, [&](long long a, long long bnd) {
    for (long long i = a; i < bnd; ++i) {
      double u[8], p[8], du[8][16];  // du[j][m] = d u_j / d theta_m
      for (int k = 0; k < P; ++k) p[k] = params[i * P + k];
      for (int k = 0; k < D; ++k) u[k] = u0[i * D + k];
      for (int j = 0; j < D; ++j)
        for (int mm = 0; mm < M; ++mm) du[j][mm] = (mm == P + j) ? 1.0 : 0.0;
      const double t0 = tspan[i * 2], tf = tspan[i * 2 + 1];
      long long n = (tf > t0) ? (long long)std::ceil((tf - t0) / dt - 1e-12) : 0;
      const double h_last = n > 0 ? tf - (t0 + double(n - 1) * dt) : 0.0;
      for (long long s = 0; s < n; ++s) {
        const double h = (s == n - 1) ? h_last : dt;
        const double t = t0 + double(s) * dt;
        double k[7][8], dk[7][8][16], U[8], dU[8][16], Ju[64], Jp[64];
        for (int st = 0; st < S; ++st) {
          for (int j = 0; j < D; ++j) {
            double acc = 0;
            for (int q = 0; q < st; ++q) acc += TA[st][q] * k[q][j];
            U[j] = u[j] + h * acc;
            for (int mm = 0; mm < M; ++mm) {
              double dacc = 0;
              for (int q = 0; q < st; ++q) dacc += TA[st][q] * dk[q][j][mm];
              dU[j][mm] = du[j][mm] + h * dacc;
            }
          }
          rhs<double>(rhs_id, U, p, t + TC[st] * h, k[st]);
          jac_u<double>(rhs_id, U, p, t + TC[st] * h, Ju);
          jac_p<double>(rhs_id, U, p, t + TC[st] * h, Jp);
          for (int j = 0; j < D; ++j)
            for (int mm = 0; mm < M; ++mm) {
              double v = (mm < P) ? Jp[j * P + mm] : 0.0;
              for (int q = 0; q < D; ++q) v += Ju[j * D + q] * dU[q][mm];
              dk[st][j][mm] = v;
            }
        }
        for (int j = 0; j < D; ++j) {
          double acc = 0;
          for (int q = 0; q < S; ++q) acc += TB[q] * k[q][j];
          double unew = u[j] + h * acc;
          for (int mm = 0; mm < M; ++mm) {
            double dacc = 0;
            for (int q = 0; q < S; ++q) dacc += TB[q] * dk[q][j][mm];
            du[j][mm] = du[j][mm] + h * dacc;
          }
          u[j] = unew;
        }
      }
      for (int mm = 0; mm < M; ++mm) {
        double g = 0;
        for (int j = 0; j < D; ++j) g += grad_out[i * D + j] * du[j][mm];
        if (mm < P) g_p[i * P + mm] = g;
        else g_u0[i * D + (mm - P)] = g;
      }
      if (u_final)
        for (int j = 0; j < D; ++j) u_final[i * D + j] = u[j];
    }
  });
  return 0;
}

int oracle_tsit5_fixed_grad(int rhs_id, long long N, const double* params, const double* u0,
                            const double* tspan, double dt, const double* grad_out,
                            double* g_p, double* g_u0, double* u_final, int nthreads) {
  return oracle_fixed_grad(rhs_id, ALG_TSIT5_FIXED, N, params, u0, tspan, dt, grad_out, g_p,
                           g_u0, u_final, nthreads);
}

}  // extern "C"
