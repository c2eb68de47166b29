"""Pins of the oracle's dense output for adaptive Tsit5 (the continuous extension defined in
oracle/dense.py) to facts fixed outside the C++ code:

* the typed constants (the oracle's, and the CUDA header's read as text) equal the 40-digit
  derivation;
* against the C++ oracle's own tableau: the order conditions of every rooted tree of order
  <= 4 hold at every theta (checked at several), b_i(1) = b_i, and the derivative is f at
  both ends (C1 across steps);
* on u' = mu u the one-step interpolation error against exp(theta mu h) falls as h^5;
* the chosen member minimises the integrated 5th-order defect along the free direction;
* the solver's dense saving: the step sequence and final state equal those of a solve
  without save times, saves at t0 / tf are the initial / final state, saves outside the
  span are NaN, and interior saves are within 10x tolerance of a tol-1e-12 reference.
"""
import numpy as np
import pytest

import oracle
import workloads

mp = pytest.importorskip("mpmath")  # the derivation needs it; the GPU machine's image lacks it
from oracle import dense  # noqa: E402

THETAS = (0.0, 0.1, 0.37, 0.5, 0.83, 1.0)


def _weights(theta, r):
    return np.array([theta * (ri[0] + theta * (ri[1] + theta * (ri[2] + theta * ri[3])))
                     for ri in r])


def _dweights(theta, r):
    return np.array([ri[0] + theta * (2 * ri[1] + theta * (3 * ri[2] + theta * 4 * ri[3]))
                     for ri in r])


def test_typed_constants_equal_the_derivation():
    np.testing.assert_allclose(oracle.tsit5_dense(), np.array(dense.derive()), rtol=1e-15,
                               atol=1e-16)


def test_kernel_constants_equal_the_derivation():
    """The CUDA path types the same coefficients independently (ts5_dense in its device
    header); read them from the source text and compare with the derivation."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2304_06835_gb300", "csrc",
                            "ens_device.cuh")).read()
    body = src[src.index("constexpr double ts5_dense("):]
    body = body[body.index("= {") + 3:body.index("};")]
    rows = re.findall(r"\{([^{}]*)\}", body)
    k = np.array([[float(x) for x in r.split(",")] for r in rows])
    assert k.shape == (7, 4)
    np.testing.assert_allclose(k, np.array(dense.derive()), rtol=1e-15, atol=1e-16)


def test_order_conditions_at_every_theta():
    c, A, b, _ = oracle.tsit5_tableau()
    A = A.copy()
    A[6] = b  # FSAL stage
    Ac = A @ c
    trees = [(np.ones(7), 1), (c, 2), (c ** 2, 3), (Ac, 6), (c ** 3, 4), (c * Ac, 8),
             (A @ c ** 2, 12), (A @ Ac, 24)]
    order = [1, 2, 3, 3, 4, 4, 4, 4]
    r = oracle.tsit5_dense()
    for th in THETAS:
        bt = _weights(th, r)
        for (phi, gamma), q in zip(trees, order):
            # coefficients up to ~90 cancel: float64 rounding of the sums is ~1e-14
            assert bt @ phi == pytest.approx(th ** q / gamma, abs=1e-13), (th, gamma)
    np.testing.assert_allclose(_weights(1.0, r), b, atol=1e-13)
    np.testing.assert_allclose(_dweights(0.0, r), np.eye(7)[0], atol=1e-13)
    np.testing.assert_allclose(_dweights(1.0, r), np.eye(7)[6], atol=1e-13)


def test_interpolation_error_on_linear_problem_is_fifth_order():
    """u' = mu u: k_i = mu U_i; the interpolant against exp(theta mu h)."""
    c, A, b, _ = oracle.tsit5_tableau()
    r = oracle.tsit5_dense()
    mu = -1.3

    def err(h):
        k = np.zeros(7)
        for i in range(7):
            Ui = 1.0 + h * (A[i, :i] @ k[:i]) if i < 6 else 1.0 + h * (b[:6] @ k[:6])
            k[i] = mu * Ui
        return max(abs(1.0 + h * (_weights(th, r) @ k) - np.exp(th * mu * h))
                   for th in (0.25, 0.5, 0.75))

    e1, e2 = err(0.2), err(0.1)
    assert 2 ** 4.6 < e1 / e2 < 2 ** 5.4, (e1, e2)


def test_chosen_member_minimises_the_fifth_order_defect():
    with mp.workdps(40):
        c, A, b = dense.tableau()
        x, null = dense.family()
        M, y = dense._constraints(c, A, b)
        # the free direction keeps every condition (order <= 4, b(1) = b, C1)
        assert max(abs(v) for v in M * null) < mp.mpf("1e-15")
        f0 = dense.defect5(x, c, A)
        for eps in ("1e-3", "-1e-3"):
            assert dense.defect5(x + mp.mpf(eps) * null, c, A) > f0


def test_dense_saving_semantics():
    P, U, T = workloads.lorenz_random(64, seed=12, t1=1.0)
    P[:, 1] = np.linspace(1.0, 9.0, 64)  # rho < 10: no chaos, so errors stay comparable
    sv = np.array([-0.5, 0.0, 0.013, 0.25, 0.5, 0.999, 1.0, 1.5])
    tol = 1e-8
    o, st, stats = oracle.solve("lorenz", "tsit5", P, U, T, abstol=tol, reltol=tol, saveat=sv,
                                dense=True)
    f, stf, statsf = oracle.solve("lorenz", "tsit5", P, U, T, abstol=tol, reltol=tol)
    ref, _, _ = oracle.solve("lorenz", "tsit5", P, U, T, abstol=1e-12, reltol=1e-12, saveat=sv)
    np.testing.assert_array_equal(stats, statsf)
    np.testing.assert_array_equal(o[:, 6], f)
    np.testing.assert_array_equal(o[:, 1], U)
    assert np.all(np.isnan(o[:, 0])) and np.all(np.isnan(o[:, 7]))
    inner = o[:, 2:6]
    assert np.all(np.abs(inner - ref[:, 2:6]) <= 10 * (tol + tol * np.abs(ref[:, 2:6])))
    # the non-dense path steps onto the save times: more steps, same answers within tolerance
    s2, _, stats2 = oracle.solve("lorenz", "tsit5", P, U, T, abstol=tol, reltol=tol, saveat=sv)
    assert np.all(stats2[:, 0] >= stats[:, 0])
