"""Seeded synthetic inputs for the ensemble workloads.

This module holds no arithmetic of the method: it only draws parameters, initial states and
time spans (NumPy ``default_rng``), so that the CUDA path, the CPU oracle, the tests and the
benchmark see the same inputs.  All arrays are float64, row-major ``[N, P]`` / ``[N, D]`` /
``[N, 2]``.

Workloads (the paper's models with the shapes and value ranges of its benchmarks):
  * ``lorenz_sweep``      -- Lorenz, sigma=10, beta=8/3, rho linearly spaced over [0, 21],
                             u0=(1,0,0), tspan [0,1] (Sec. 6.4 sweep; Appendix, Lorenz problem).
  * ``lorenz_random``     -- Lorenz, rho~U[0,28], sigma~U[8,12], beta~U[2,3], u0=(1,0,0).
  * ``robertson_random``  -- Robertson, k = (0.04, 3e7, 1e4) each times a log-uniform factor in
                             [0.9, 1.1], u0=(1,0,0), tspan [0, 1e5] (Appendix, Robertson equation).
  * ``gbm_random``        -- geometric Brownian motion dX = mu X dt + sigma X dW, mu~U[-0.5,0.5],
                             sigma~U[0.1,0.5], X0=1, tspan [0,1] (Appendix, linear SDE).
  * ``uneven_batch``      -- the three above mixed: Lorenz with tf~U[1,100], Robertson, GBM.
  * ``adjoint_targets``   -- targets u_target ~ N(0, 5^2) per component.
  * ``surrogate_inputs``  -- (sigma, rho, beta, u0) with u0~U[-5,5]^3, optionally with a share of
                             samples from a 1.25x enlarged box.
  * ``crn_grid``          -- sigma-factor CRN SDE, p = (S, D, tau, nu0, n, eta): k values of each
                             parameter drawn uniformly in its range (S, D, tau in [0.1, 100],
                             nu0 in [0.01, 0.2], n in [2, 4], eta in [0.001, 0.1]), all k^6
                             combinations (the Cartesian product), u0 = (nu0, nu0, nu0, nu0),
                             tspan [0, 1000] (Appendix, CRN model and its parameter table).
  * ``crn_random``        -- the same ranges, each trajectory's parameters drawn independently.
  * ``stiff``             -- the paper's stiff test models with their printed initial states and
                             spans: Orego (k = (77.27, 8.375e-6, 0.161), y0 = (1, 2, 3), [0, 30]),
                             HIRES (its 12 distinct constants, y0 = (1, 0, ..., 0, 0.0057),
                             [0, 321.8122]), POLLU (k1..k25 as printed, y0 as printed, [0, 60]).
                             Orego and POLLU: each trajectory scales every constant by its own
                             log-uniform factor in [0.9, 1.1] (the Robertson ensemble's recipe).
                             HIRES: its loss constants are sums of its gain constants (8.75 =
                             0.43 + 8.32, 10.03 = 8.32 + 1.71, ...), so all 12 share one factor
                             (which keeps every sum) and the nonlinear rate 280 takes a second.
  * ``ball``              -- bouncing ball, p = (g, e) with g = 9.8 and the coefficient of
                             restitution e ~ U[0.7, 0.95] per trajectory, u0 = (50, 0) (a drop
                             from 50 m at rest), tspan [0, 15] (Appendix, bouncing-ball problem;
                             e >= 0.65 keeps the bounces' accumulation point after t = 15).
"""
from __future__ import annotations

import numpy as np

LORENZ_BOX = np.array([[8.0, 12.0], [0.0, 28.0], [2.0, 3.0]])  # sigma, rho, beta
U0_BOX = np.array([[-5.0, 5.0]] * 3)
ROBERTSON_K0 = np.array([0.04, 3e7, 1e4])
CRN_BOX = np.array([[0.1, 100.0], [0.1, 100.0], [0.1, 100.0], [0.01, 0.2], [2.0, 4.0],
                    [0.001, 0.1]])  # S, D, tau, nu0, n, eta


def lorenz_sweep(N: int = 1024, t1: float = 1.0):
    rho = 21.0 * np.arange(N, dtype=np.float64) / max(N - 1, 1)
    params = np.stack([np.full(N, 10.0), rho, np.full(N, 8.0 / 3.0)], axis=1)
    u0 = np.tile(np.array([1.0, 0.0, 0.0]), (N, 1))
    tspan = np.tile(np.array([0.0, t1]), (N, 1))
    return params, u0, tspan


def lorenz_random(N: int = 1 << 20, seed: int = 2, t1: float = 10.0):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.0, 28.0, N)
    sigma = rng.uniform(8.0, 12.0, N)
    beta = rng.uniform(2.0, 3.0, N)
    params = np.stack([sigma, rho, beta], axis=1)
    u0 = np.tile(np.array([1.0, 0.0, 0.0]), (N, 1))
    tspan = np.tile(np.array([0.0, t1]), (N, 1))
    return params, u0, tspan


def robertson_random(N: int = 1 << 18, seed: int = 3, t1: float = 1e5):
    rng = np.random.default_rng(seed)
    fac = np.exp(rng.uniform(np.log(0.9), np.log(1.1), (N, 3)))
    params = ROBERTSON_K0[None, :] * fac
    u0 = np.tile(np.array([1.0, 0.0, 0.0]), (N, 1))
    tspan = np.tile(np.array([0.0, t1]), (N, 1))
    return params, u0, tspan


def gbm_random(N: int = 300_000, seed: int = 4, t1: float = 1.0):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-0.5, 0.5, N)
    sig = rng.uniform(0.1, 0.5, N)
    params = np.stack([mu, sig], axis=1)
    u0 = np.ones((N, 1))
    tspan = np.tile(np.array([0.0, t1]), (N, 1))
    return params, u0, tspan


def uneven_batch(n_lorenz: int = 500_000, n_rober: int = 200_000, n_gbm: int = 300_000,
                 seed: int = 4):
    """Mixed batch: returns dict name -> (params, u0, tspan)."""
    rng = np.random.default_rng(seed)
    s1, s2, s3 = rng.integers(0, 2**31 - 1, 3)
    lp, lu, lt = lorenz_random(n_lorenz, int(s1))
    lt[:, 1] = np.random.default_rng(int(s1) + 1).uniform(1.0, 100.0, n_lorenz)
    rp, ru, rt = robertson_random(n_rober, int(s2))
    gp, gu, gt = gbm_random(n_gbm, int(s3))
    return {"lorenz": (lp, lu, lt), "robertson": (rp, ru, rt), "gbm": (gp, gu, gt)}


def adjoint_targets(N: int = 65536, seed: int = 5):
    rng = np.random.default_rng(seed + 1000)
    return rng.normal(0.0, 5.0, (N, 3))


def surrogate_inputs(N: int, seed: int, outside_share: float = 0.0, enlarge: float = 1.25):
    """x [N, 6] = (sigma, rho, beta, u0_1, u0_2, u0_3).  A share of rows is drawn from the box
    enlarged by `enlarge` about its centre (to exercise the out-of-box fallback)."""
    rng = np.random.default_rng(seed)
    box = np.concatenate([LORENZ_BOX, U0_BOX], axis=0)
    lo, hi = box[:, 0], box[:, 1]
    x = rng.uniform(lo, hi, (N, 6))
    n_out = int(round(outside_share * N))
    if n_out:
        c, r = (lo + hi) / 2, (hi - lo) / 2 * enlarge
        x[N - n_out:] = rng.uniform(c - r, c + r, (n_out, 6))
        perm = rng.permutation(N)
        x = x[perm]
    return x


def surrogate_box():
    return np.concatenate([LORENZ_BOX, U0_BOX], axis=0)


def _crn_problem(p: np.ndarray, t1: float):
    N = p.shape[0]
    u0 = np.repeat(p[:, 3:4], 4, axis=1)
    tspan = np.zeros((N, 2))
    tspan[:, 1] = t1
    return p, u0, tspan


def crn_grid(k: int = 10, seed: int = 8, t1: float = 1000.0):
    """Cartesian product of k uniform draws per parameter: k**6 trajectories."""
    rng = np.random.default_rng(seed)
    axes = [np.sort(rng.uniform(lo, hi, k)) for lo, hi in CRN_BOX]
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 6)
    return _crn_problem(np.ascontiguousarray(grid), t1)


def crn_random(N: int, seed: int = 9, t1: float = 1000.0):
    rng = np.random.default_rng(seed)
    p = rng.uniform(CRN_BOX[:, 0], CRN_BOX[:, 1], size=(N, 6))
    return _crn_problem(p, t1)


def ball(N: int, seed: int = 10, t1: float = 15.0, x0: float = 50.0):
    rng = np.random.default_rng(seed)
    p = np.stack([np.full(N, 9.8), rng.uniform(0.7, 0.95, N)], axis=1)
    u0 = np.tile([x0, 0.0], (N, 1))
    tspan = np.zeros((N, 2))
    tspan[:, 1] = t1
    return p, u0, tspan


OREGO_K = [77.27, 8.375e-6, 0.161]
HIRES_C = [1.71, 0.43, 8.32, 0.0007, 8.75, 10.03, 0.035, 1.12, 1.745, 280.0, 0.69, 1.81]
POLLU_K = [0.35, 26.6, 12300.0, 0.00086, 0.00082, 15000.0, 0.00013, 24000.0, 16500.0, 9000.0,
           0.022, 12000.0, 1.88, 16300.0, 4.8e6, 0.00035, 0.0175, 1.0e8, 4.44e11, 1240.0, 2.1,
           5.78, 0.0474, 1780.0, 3.12]
STIFF = {
    "orego": (OREGO_K, [1.0, 2.0, 3.0], 30.0),
    "hires": (HIRES_C, [1.0, 0, 0, 0, 0, 0, 0, 0.0057], 321.8122),
    "pollu": (POLLU_K, [0.0, 0.2, 0.0, 0.04, 0.0, 0.0, 0.1, 0.3, 0.017, 0.0, 0.0, 0.0, 0.0, 0.0,
                        0.0, 0.0, 0.007, 0.0, 0.0, 0.0], 60.0),
}


def stiff(model: str, N: int, seed: int = 11, t1: float | None = None):
    k0, y0, tf = STIFF[model]
    rng = np.random.default_rng(seed)
    lo, hi = np.log(0.9), np.log(1.1)
    if model == "hires":
        k = np.asarray(k0) * np.exp(rng.uniform(lo, hi, (N, 1)))
        k[:, 9] *= np.exp(rng.uniform(lo, hi, N))
    else:
        k = np.asarray(k0) * np.exp(rng.uniform(lo, hi, (N, len(k0))))
    u0 = np.tile(y0, (N, 1)).astype(np.float64)
    tspan = np.zeros((N, 2))
    tspan[:, 1] = tf if t1 is None else t1
    return k, u0, tspan
