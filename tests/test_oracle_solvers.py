"""Pins of the oracle's integrators to closed forms, invariants, observed orders and library
solvers (scipy DOP853 / Radau run here as independent references).

Paper passages: explicit RK steps and the embedded estimate (Sec. 3.1), Rosenbrock step
(Sec. 3.2.1), the Lorenz and Robertson models (Appendix), fixed stepping with dt = 0.001
over [0,1] -- 1000 steps (Appendix, Lorenz problem).
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
import workloads


def lorenz_f(t, y, s, r, b):
    return [s * (y[1] - y[0]), y[0] * (r - y[2]) - y[1], y[0] * y[1] - b * y[2]]


def rober_f(t, y, k1, k2, k3):
    return [-k1 * y[0] + k3 * y[1] * y[2], k1 * y[0] - k2 * y[1] ** 2 - k3 * y[1] * y[2],
            k2 * y[1] ** 2]


# ---------------------------------------------------------------------------- models
def test_rhs_worked_values():
    # Lorenz at u=(1,2,3), (sigma,rho,beta)=(10,28,8/3): (10*(2-1), 28*1-2-1*3, 1*2-8/3*3)
    np.testing.assert_allclose(oracle.rhs_eval("lorenz", [1, 2, 3], [10, 28, 8 / 3]),
                               [10.0, 23.0, -6.0], rtol=1e-15)
    # Robertson at u=(1,0,0): only the k1 reaction runs
    np.testing.assert_allclose(oracle.rhs_eval("robertson", [1, 0, 0], [0.04, 3e7, 1e4]),
                               [-0.04, 0.04, 0.0], rtol=1e-15)
    np.testing.assert_allclose(oracle.rhs_eval("gbm", [2.0], [1.5, 0.01]), [3.0])


def test_robertson_conserves_mass_and_lorenz_divergence():
    rng = np.random.default_rng(0)
    for _ in range(20):
        u = rng.uniform(0, 1, 3)
        k = rng.uniform(0.5, 2, 3) * workloads.ROBERTSON_K0
        assert abs(oracle.rhs_eval("robertson", u, k).sum()) <= 1e-9 * np.abs(k).max()
        Ju, _ = oracle.jacobians("robertson", u, k)
        np.testing.assert_allclose(Ju.sum(axis=0), 0, atol=1e-7)  # c^T J = 0
        p = [rng.uniform(8, 12), rng.uniform(0, 28), rng.uniform(2, 3)]
        Jl, _ = oracle.jacobians("lorenz", rng.normal(size=3) * 5, p)
        assert abs(np.trace(Jl) - (-p[0] - 1 - p[2])) < 1e-13  # div f = -(sigma + 1 + beta)


@pytest.mark.parametrize("rhs", ["lorenz", "robertson", "gbm"])
def test_jacobians_central_differences(rhs):
    rng = np.random.default_rng(1)
    D, P = oracle.DIMS[oracle.RHS[rhs]]
    for _ in range(5):
        u = rng.uniform(0.1, 2, D)
        p = rng.uniform(0.5, 2, P) * (workloads.ROBERTSON_K0 * 1e-3 if rhs == "robertson" else 1)
        Ju, Jp = oracle.jacobians(rhs, u, p)
        for j in range(D):
            e = np.zeros(D)
            hh = 1e-3 * max(1, abs(u[j]))  # f is at most quadratic: central differences exact
            e[j] = hh
            fp, fm = oracle.rhs_eval(rhs, u + e, p), oracle.rhs_eval(rhs, u - e, p)
            fd = (fp - fm) / (2 * hh)
            roundoff = 8 * np.finfo(float).eps * np.abs(np.concatenate([fp, fm])).max() / hh
            np.testing.assert_allclose(Ju[:, j], fd, rtol=1e-9, atol=roundoff + 1e-14)
        for m in range(P):
            e = np.zeros(P)
            hh = 0.1 * abs(p[m])  # f is linear in p
            e[m] = hh
            fp, fm = oracle.rhs_eval(rhs, u, p + e), oracle.rhs_eval(rhs, u, p - e)
            fd = (fp - fm) / (2 * hh)
            roundoff = 8 * np.finfo(float).eps * np.abs(np.concatenate([fp, fm])).max() / hh
            np.testing.assert_allclose(Jp[:, m], fd, rtol=1e-9, atol=roundoff + 1e-14)


def test_lu_solve_matches_numpy():
    rng = np.random.default_rng(2)
    for D in (1, 2, 3, 5, 8):
        for _ in range(20):
            W = rng.normal(size=(D, D))
            b = rng.normal(size=D)
            np.testing.assert_allclose(oracle.lu_solve(W, b), np.linalg.solve(W, b),
                                       rtol=1e-9, atol=1e-12)
    # needs pivoting: zero leading entry
    W = np.array([[0.0, 1.0, 2.0], [1.0, 1.0, 0.0], [2.0, 0.0, 1.0]])
    b = np.array([1.0, 2.0, 3.0])
    np.testing.assert_allclose(oracle.lu_solve(W, b), np.linalg.solve(W, b), rtol=1e-13)
    # near-singular but well-posed under pivoting
    W = np.array([[1e-12, 1.0, 0.0], [1.0, 1.0, 1.0], [0.0, 1.0, 3.0]])
    np.testing.assert_allclose(oracle.lu_solve(W, b), np.linalg.solve(W, b), rtol=1e-10)


# ---------------------------------------------------------------------------- closed forms
def _stab_poly(c, A, b, z):
    # R(z) = 1 + z b^T (I - zA)^{-1} 1
    s = A.shape[0]
    return 1 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))


@pytest.mark.parametrize("mu", [-1.0, -0.3, 0.5])
def test_linear_fixed_step_equals_stability_function_power(mu):
    """u' = mu u (the GBM drift): n fixed Tsit5 steps give R(h mu)^n u0 exactly, and RK4 gives
    (1 + z + z^2/2 + z^3/6 + z^4/24)^n."""
    c, A, b, _ = oracle.tsit5_tableau()
    h, n = 1e-2, 100
    P = np.array([[mu, 0.3]])
    u0 = np.array([[1.7]])
    ts = np.array([[0.0, 1.0]])
    out, st, stt = oracle.solve("gbm", "tsit5_fixed", P, u0, ts, dt=h)
    z = h * mu
    exact_map = _stab_poly(c, A, b, z) ** n * 1.7
    assert abs(out[0, 0] - exact_map) <= 1e-13 * abs(exact_map)
    assert abs(out[0, 0] - 1.7 * math.exp(mu)) <= 1e-11
    assert st[0] == 0 and stt[0, 0] == n and stt[0, 2] == 1 + 6 * n
    out4, _, _ = oracle.solve("gbm", "rk4", P, u0, ts, dt=h)
    r4 = 1 + z + z * z / 2 + z**3 / 6 + z**4 / 24
    assert abs(out4[0, 0] - 1.7 * r4**n) <= 1e-13 * abs(out4[0, 0])


def test_lorenz_rho0_closed_form():
    """rho = 0, u0 = (1,0,0): y2, y3 stay exactly 0 and y1(1) = R(-sigma h)^1000 (1000 steps)."""
    c, A, b, _ = oracle.tsit5_tableau()
    P, U, T = workloads.lorenz_sweep(4)
    out, st, stt = oracle.solve("lorenz", "tsit5_fixed", P, U, T, dt=1e-3)
    assert stt[0, 0] == 1000 and np.all(stt[:, 0] == 1000)
    assert out[0, 1] == 0.0 and out[0, 2] == 0.0
    r = _stab_poly(c, A, b, -10 * 1e-3) ** 1000
    assert abs(out[0, 0] - r) < 1e-14
    assert abs(out[0, 0] - math.exp(-10.0)) < 1e-12


# ---------------------------------------------------------------------------- orders
def _lorenz_ref(p, u0, t1):
    sol = solve_ivp(lorenz_f, (0, t1), u0, method="DOP853", rtol=1e-13, atol=1e-13, args=tuple(p))
    return sol.y[:, -1]


def test_fixed_step_convergence_orders():
    p = [10.0, 21.0, 8 / 3]
    u0 = [1.0, 0.0, 0.0]
    ref = _lorenz_ref(p, u0, 1.0)
    for alg, order in (("tsit5_fixed", 5), ("rk4", 4)):
        errs = []
        dts = [1 / 100, 1 / 200, 1 / 400, 1 / 800]
        for dt in dts:
            out, _, _ = oracle.solve("lorenz", alg, [p], [u0], [[0, 1]], dt=dt)
            errs.append(np.abs(out[0] - ref).max())
        slopes = np.diff(np.log(errs)) / np.diff(np.log(dts))
        # the last two halvings are in the asymptotic regime
        assert np.all(np.abs(slopes[1:] - order) < 0.3), (alg, slopes, errs)


def _one_step_errors(alg, rhs, u, p, hs, exact):
    e_main, e_emb = [], []
    for h in hs:
        un, err = oracle.step(rhs, alg, u, p, 0.0, h)
        ex = exact(h)
        e_main.append(np.abs(un - ex).max())
        e_emb.append(np.abs(un + err - ex).max())
    return np.array(e_main), np.array(e_emb)


def test_local_error_orders_tsit5_and_embedded():
    """Local error of u_{n+1} is O(h^6); of the embedded solution u_{n+1} + E is O(h^5)."""
    p = [10.0, 21.0, 8 / 3]
    u = np.array([1.0, 2.0, 3.0])
    hs = np.array([0.02, 0.01, 0.005])
    exact = lambda h: solve_ivp(lorenz_f, (0, h), u, method="DOP853", rtol=1e-14, atol=1e-15,
                                args=tuple(p)).y[:, -1]
    em, ee = _one_step_errors("tsit5", "lorenz", u, p, hs, exact)
    s_main = np.diff(np.log(em)) / np.diff(np.log(hs))
    s_emb = np.diff(np.log(ee)) / np.diff(np.log(hs))
    assert np.all(s_main > 5.4), s_main
    assert np.all(np.abs(s_emb - 5) < 0.4), s_emb


def test_rosenbrock23_orders():
    """ode23s: u_{n+1} is order 2 (local error h^3); u_{n+1} + E is order 3 (local h^4)."""
    k = [0.04, 3e1, 1e1]  # mildly stiff so the asymptotic regime is reachable
    u = np.array([0.8, 0.1, 0.1])
    hs = np.array([0.04, 0.02, 0.01])
    exact = lambda h: solve_ivp(rober_f, (0, h), u, method="Radau", rtol=1e-13, atol=1e-15,
                                args=tuple(k)).y[:, -1]
    em, ee = _one_step_errors("ros23", "robertson", u, k, hs, exact)
    s_main = np.diff(np.log(em)) / np.diff(np.log(hs))
    s_emb = np.diff(np.log(ee)) / np.diff(np.log(hs))
    assert np.all(np.abs(s_main - 3) < 0.3), s_main
    assert np.all(np.abs(s_emb - 4) < 0.4), s_emb


def test_rosenbrock23_scalar_map_and_L_stability():
    """u' = mu u: the step map is a rational function R(z) with R(z) = 1 + z + z^2/2 + O(z^3)
    and R(z) -> 0 as z -> -inf (L-stability, Sec. 5.2.1 'L-Stable Rosenbrock-W')."""
    for z in (1e-3, 2e-3):
        un, _ = oracle.step("gbm", "ros23", [1.0], [z, 0.0], 0.0, 1.0)
        assert abs(un[0] - (1 + z + z * z / 2)) < 2 * z**3
    r = [abs(oracle.step("gbm", "ros23", [1.0], [-10.0**e, 0.0], 0.0, 1.0)[0][0])
         for e in (2, 4, 6, 8)]
    assert r[-1] < 1e-6 and all(r[i + 1] < r[i] for i in range(3))


# ---------------------------------------------------------------------------- adaptive
def test_adaptive_tsit5_within_10x_tolerance():
    P, U, T = workloads.lorenz_random(64, seed=11, t1=1.0)
    for tol in (1e-6, 1e-8):
        out, st, stt = oracle.solve("lorenz", "tsit5", P, U, T, abstol=tol, reltol=tol)
        assert np.all(st == 0)
        for i in range(0, 64, 4):
            ref = _lorenz_ref(P[i], U[i], 1.0)
            assert np.all(np.abs(out[i] - ref) <= 10 * (tol + tol * np.abs(ref))), (i, out[i], ref)


def test_adaptive_step_count_scaling():
    """Accepted steps grow like tol^(-1/5) for a 5th-order pair: x10^5 in tol -> ~x10."""
    P, U, T = workloads.lorenz_random(32, seed=12, t1=1.0)
    _, _, s5 = oracle.solve("lorenz", "tsit5", P, U, T, abstol=1e-5, reltol=1e-5)
    _, _, s10 = oracle.solve("lorenz", "tsit5", P, U, T, abstol=1e-10, reltol=1e-10)
    ratio = s10[:, 0].sum() / s5[:, 0].sum()
    assert 6 < ratio < 16, ratio
    assert s5[:, 1].sum() < 0.25 * s5[:, 0].sum()


def test_adaptive_reference_tol12_matches_scipy():
    P, U, T = workloads.lorenz_random(8, seed=13, t1=10.0)
    out, st, _ = oracle.solve("lorenz", "tsit5", P, U, T, abstol=1e-12, reltol=1e-12)
    for i in range(8):
        if P[i, 1] < 10:
            ref = _lorenz_ref(P[i], U[i], 10.0)
            assert np.all(np.abs(out[i] - ref) <= 1e-9 * (1 + np.abs(ref)))


def test_saveat_hits_times_and_matches_reference():
    P, U, T = workloads.lorenz_random(4, seed=14, t1=1.0)
    sv = [0.0, 0.25, 0.5, 1.0, 1.5]
    out, st, _ = oracle.solve("lorenz", "tsit5", P, U, T, abstol=1e-10, reltol=1e-10, saveat=sv)
    assert out.shape == (4, 5, 3)
    np.testing.assert_array_equal(out[:, 0], U)
    assert np.all(np.isnan(out[:, 4]))  # beyond tf
    for i in range(4):
        sol = solve_ivp(lorenz_f, (0, 1), U[i], method="DOP853", rtol=1e-13, atol=1e-13,
                        args=tuple(P[i]), t_eval=[0.25, 0.5, 1.0])
        np.testing.assert_allclose(out[i, 1:4], sol.y.T, atol=1e-7, rtol=1e-7)


def test_fixed_saveat_grid():
    P, U, T = workloads.lorenz_sweep(3)
    sv = [0.0, 0.5, 1.0]
    out, _, _ = oracle.solve("lorenz", "tsit5_fixed", P, U, T, dt=1e-3, saveat=sv)
    fin, _, _ = oracle.solve("lorenz", "tsit5_fixed", P, U, T, dt=1e-3)
    half, _, _ = oracle.solve("lorenz", "tsit5_fixed", P, U, T * 0.5, dt=1e-3)
    np.testing.assert_array_equal(out[:, 0], U)
    np.testing.assert_array_equal(out[:, 2], fin)
    np.testing.assert_array_equal(out[:, 1], half)


def test_robertson_ros23_mass_and_radau_reference():
    P, U, T = workloads.robertson_random(6, seed=15)
    sv = np.logspace(-4, 5, 10)
    tol = 1e-6
    out, st, stt = oracle.solve("robertson", "ros23", P, U, T, abstol=tol, reltol=tol, dt0=1e-4,
                                saveat=sv)
    assert np.all(st == 0)
    steps = stt[:, 0] + stt[:, 1]
    mass = out.sum(axis=2)
    assert np.all(np.abs(mass - 1) <= 1e-13 * steps[:, None] + 1e-15)
    for i in range(6):
        sol = solve_ivp(rober_f, (0, 1e5), U[i], method="Radau", rtol=1e-12, atol=1e-14,
                        args=tuple(P[i]), t_eval=sv)
        ref = sol.y.T
        assert np.all(np.abs(out[i] - ref) <= 10 * (tol + tol * np.abs(ref))), i


def test_status_codes():
    P, U, T = workloads.lorenz_random(2, seed=16, t1=10.0)
    _, st, stt = oracle.solve("lorenz", "tsit5", P, U, T, abstol=1e-8, reltol=1e-8, maxiters=10)
    assert np.all(st == 1) and np.all(stt[:, 0] + stt[:, 1] == 10)
    Pn = P.copy()
    Pn[0, 0] = np.nan
    _, st, _ = oracle.solve("lorenz", "tsit5", Pn, U, T, abstol=1e-8, reltol=1e-8)
    assert st[0] == 3 and st[1] == 0
    _, st, _ = oracle.solve("lorenz", "tsit5_fixed", Pn, U, T, dt=1e-2)
    assert st[0] == 3 and st[1] == 0
    # t0 == tf: zero steps, u0 returned
    out, st, stt = oracle.solve("lorenz", "tsit5", P, U, np.zeros((2, 2)))
    np.testing.assert_array_equal(out, U)
    assert np.all(stt[:, 0] == 0)


def test_fp32_mode_close_to_fp64():
    P, U, T = workloads.lorenz_sweep(64)
    P32 = P.astype(np.float32).astype(np.float64)
    o64, _, _ = oracle.solve("lorenz", "tsit5_fixed", P32, U, T, dt=1e-3)
    o32, _, _ = oracle.solve("lorenz", "tsit5_fixed", P32, U, T, dt=1e-3, precision="f32")
    # state-vector relative error (the reading of the 1e-5 FP32 bound used for parity)
    err = np.abs(o32 - o64).max(axis=1)
    scale = np.maximum(np.abs(o64).max(axis=1), 1)
    assert np.all(err <= 1e-5 * scale)
