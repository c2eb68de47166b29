"""Pins of the oracle's stiff test models (Appendix: OREGO, HIRES, POLLU) and of its
Rosenbrock23 at dimensions 3, 8 and 20:

* every analytic Jacobian equals central finite differences of f;
* POLLU's printed equations equal the sum over its 25 mass-action reactions (an independent
  reading of the same mechanism);
* conservation: HIRES keeps y7 + y8, and POLLU keeps every left null vector of its
  stoichiometry (computed from the reaction table with numpy), along the whole solution;
* Rosenbrock23 at a tight tolerance agrees with SciPy's Radau IIA (a different method and
  implementation) on each model.
"""
import numpy as np
import pytest

import oracle
import workloads

MODELS = ("orego", "hires", "pollu")


@pytest.mark.parametrize("model", MODELS)
def test_jacobian_matches_finite_differences(model):
    P, U, _ = workloads.stiff(model, 3, seed=2)
    rng = np.random.default_rng(1)
    for i in range(3):
        y = U[i] + rng.uniform(0.01, 1.0, U.shape[1]) * (10.0 if model == "orego" else 0.1)
        J = oracle.jac_u(model, y, P[i])
        Jfd = np.empty_like(J)
        for j in range(len(y)):
            h = 1e-6 * max(1.0, abs(y[j]))
            yp, ym = y.copy(), y.copy()
            yp[j] += h
            ym[j] -= h
            Jfd[:, j] = (oracle.rhs_eval(model, yp, P[i]) - oracle.rhs_eval(model, ym, P[i])) / (2 * h)
        scale = np.maximum(np.abs(J).max(axis=1, keepdims=True), 1e-300)
        assert np.all(np.abs(J - Jfd) <= 1e-6 * scale + 1e-9), model


def test_pollu_printed_equations_equal_the_reaction_sum():
    P, _, _ = workloads.stiff("pollu", 4, seed=3)
    rng = np.random.default_rng(3)
    for i in range(4):
        y = rng.uniform(0.0, 0.5, 20)
        a = oracle.rhs_eval("pollu", y, P[i])
        b = oracle.pollu_reaction_sum(y, P[i])
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13 * np.abs(b).max())


def _pollu_stoichiometry():
    """nu [20, 25] from the reaction-sum form: column j = f for k = e_j, y = reactants 1."""
    nu = np.zeros((20, 25))
    for j in range(25):
        k = np.zeros(25)
        k[j] = 1.0
        nu[:, j] = oracle.pollu_reaction_sum(np.ones(20), k)
    return nu


def test_conservation_laws_hold_along_the_solution():
    P, U, T = workloads.stiff("hires", 8, seed=4)
    sv = np.linspace(0.0, T[0, 1], 7)
    out, st, _ = oracle.solve("hires", "ros23", P, U, T, abstol=1e-9, reltol=1e-9, dt0=1e-6,
                              saveat=sv)
    assert np.all(st == 0)
    np.testing.assert_allclose(out[:, :, 6] + out[:, :, 7], 0.0057, rtol=1e-10)
    nu = _pollu_stoichiometry()
    _, s, vt = np.linalg.svd(nu.T)
    C = vt[np.sum(s > 1e-10):]  # left null space of nu: c^T nu = 0
    assert C.shape[0] >= 1
    P, U, T = workloads.stiff("pollu", 8, seed=5)
    sv = np.linspace(0.0, 60.0, 7)
    out, st, _ = oracle.solve("pollu", "ros23", P, U, T, abstol=1e-10, reltol=1e-8, dt0=1e-8,
                              saveat=sv)
    assert np.all(st == 0)
    inv = out @ C.T  # [N, S, n_laws]
    np.testing.assert_allclose(inv, inv[:, :1, :].repeat(len(sv), axis=1), atol=1e-10)


@pytest.mark.parametrize("model,tol", [("orego", 1e-5), ("hires", 1e-6), ("pollu", 1e-6)])
def test_rosenbrock23_agrees_with_scipy_radau(model, tol):
    integrate = pytest.importorskip("scipy.integrate")
    P, U, T = workloads.stiff(model, 2, seed=6)
    out, st, _ = oracle.solve(model, "ros23", P, U, T, abstol=1e-10, reltol=1e-9, dt0=1e-8)
    assert np.all(st == 0)
    for i in range(2):
        r = integrate.solve_ivp(lambda t, y: oracle.rhs_eval(model, y, P[i]), (0.0, T[i, 1]),
                                U[i], method="Radau", rtol=1e-11, atol=1e-13,
                                jac=lambda t, y: oracle.jac_u(model, y, P[i]))
        ref = r.y[:, -1]
        scale = np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max())
        assert np.all(np.abs(out[i] - ref) <= tol * scale), (model, out[i], ref)
