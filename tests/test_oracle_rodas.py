"""Pins of the oracle's Rodas4 and Rodas5P (Sec. 5.2.1: GPURodas4, Hairer-Wanner; GPURodas5P,
Steinebach 2023), stiffly accurate Rosenbrock methods of orders 4(3) and 5(4).

The oracle steps the standard form (I - h gamma J) k_i = h f(y + sum alpha_ij k_j)
+ h J sum gamma_ij k_j, y1 = y + sum b_j k_j, converted from the published transformed
coefficients.  Pinned against:

* the Rosenbrock order conditions, generated here from rooted trees (Hairer-Wanner II, IV.7):
  elementary weights as for Runge-Kutta, except that a vertex with a single child weighs by
  alpha + Gamma (the diagonal gamma included); b satisfies every condition of order <= p and
  bhat every one of order <= p - 1, and neither satisfies all of the next order;
* numbers the publications print besides (a, C): the nodes c_i = sum_j alpha_ij and the sums
  d_i = sum_j gamma_ij (the coefficients of the time derivative);
* stiff accuracy (b = last row of alpha + Gamma, c_s = 1) and L-stability: on u' = mu u the
  step map R(z) matches e^z at least to O(z^(p+1)) and tends to 0 as z -> -inf with
  |R| <= 1 on the negative axis;
* the observed local error orders p + 1 and p on Lorenz (exact Jacobian), against DOP853;
* Robertson over [0, 1e5] at tolerance 1e-6: within 10x the tolerance of SciPy's Radau at
  1e-12, with y1 + y2 + y3 = 1 kept to round-off (the linear invariant, c^T f = 0);
* a planted mistake in the step (the J sum gamma_ij k_j term dropped) breaks the order test.
"""
import itertools

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle

METHODS = {"rodas4": (4, 3), "rodas5p": (5, 4)}
NODES = {"rodas4": [0.0, 0.386, 0.21, 0.63, 1.0, 1.0],
         "rodas5p": [0.0, 0.6358126895828704, 0.4095798393397535, 0.9769306725060716,
                     0.4288403609558664, 1.0, 1.0, 1.0]}
DSUMS = {"rodas4": [0.25, -0.1043, 0.1035, -0.0362, 0.0, 0.0],
         "rodas5p": [0.21193756319429014, -0.42387512638858027, -0.3384627126235924,
                     1.8046452872882734, 2.325825639765069, 0.0, 0.0, 0.0]}


def rooted_trees(n):
    if n == 1:
        return [()]
    out = set()

    def parts(m, maxpart):
        if m == 0:
            yield []
            return
        for k in range(min(m, maxpart), 0, -1):
            for rest in parts(m - k, k):
                yield [k] + rest

    for sizes in parts(n - 1, n - 1):
        for combo in itertools.product(*[rooted_trees(s) for s in sizes]):
            out.add(tuple(sorted(combo)))
    return sorted(out)


def size(t):
    return 1 + sum(size(c) for c in t)


def density(t):
    g = size(t)
    for c in t:
        g *= density(c)
    return g


def weight(t, alpha, beta):
    """Elementary weights of a Rosenbrock method: a root with one child multiplies by
    beta = alpha + Gamma (the Jacobian terms), with several children by alpha."""
    if len(t) == 0:
        return np.ones(alpha.shape[0])
    if len(t) == 1:
        return beta @ weight(t[0], alpha, beta)
    v = np.ones(alpha.shape[0])
    for c in t:
        v = v * (alpha @ weight(c, alpha, beta))
    return v


def residuals(vec, alpha, beta, n):
    return [abs(vec @ weight(t, alpha, beta) - 1.0 / density(t)) for t in rooted_trees(n)]


@pytest.mark.parametrize("alg", sorted(METHODS))
def test_order_conditions(alg):
    p, ph = METHODS[alg]
    g, alpha, G, b, bh = oracle.rosenbrock_tableau(alg)
    np.testing.assert_allclose(np.diag(G), g, rtol=1e-15)
    assert np.all(np.triu(G, 1) == 0)
    assert np.allclose(np.triu(alpha), 0)
    beta = alpha + G
    for n in range(1, p + 1):
        assert max(residuals(b, alpha, beta, n)) < 1e-12, (alg, n)
    for n in range(1, ph + 1):
        assert max(residuals(bh, alpha, beta, n)) < 1e-12, (alg, n)
    assert max(residuals(b, alpha, beta, p + 1)) > 1e-4
    assert max(residuals(bh, alpha, beta, ph + 1)) > 1e-4
    # printed nodes and time-derivative sums; stiff accuracy
    np.testing.assert_allclose(alpha.sum(axis=1), NODES[alg], atol=1e-14)
    np.testing.assert_allclose(G.sum(axis=1), DSUMS[alg], atol=1e-13)
    np.testing.assert_allclose(b, alpha[-1] + G[-1], atol=1e-15)
    np.testing.assert_allclose(bh, alpha[-1], atol=1e-15)


@pytest.mark.parametrize("alg", sorted(METHODS))
def test_scalar_map_and_L_stability(alg):
    p, _ = METHODS[alg]
    # R(z) - e^z = O(z^(p+1)): halving z divides the difference by at least ~2^(p+1)
    # (Rodas5P's R matches e^z one order further: the linear conditions hold to order 6)
    d = [abs(oracle.step("gbm", alg, [1.0], [z, 0.0], 0.0, 1.0)[0][0] - np.exp(z))
         for z in (0.16, 0.08)]
    assert np.log2(d[0] / d[1]) > p + 1 - 0.3, d
    r = [oracle.step("gbm", alg, [1.0], [-10.0 ** e, 0.0], 0.0, 1.0)[0][0] for e in range(0, 9)]
    assert all(abs(x) <= 1.0 for x in r)
    assert abs(r[-1]) < 1e-6


def lorenz_f(t, u, s, r, b):
    return [s * (u[1] - u[0]), u[0] * (r - u[2]) - u[1], u[0] * u[1] - b * u[2]]


def local_errors(alg, hs):
    p = [10.0, 21.0, 8 / 3]
    u = np.array([1.0, 2.0, 3.0])
    em, ee = [], []
    for h in hs:
        ex = solve_ivp(lorenz_f, (0, h), u, method="DOP853", rtol=1e-14, atol=1e-15,
                       args=tuple(p)).y[:, -1]
        un, err = oracle.step("lorenz", alg, u, p, 0.0, h)
        em.append(np.abs(un - ex).max())
        ee.append(np.abs(un - err - ex).max())  # the embedded solution is y1 - E
    return np.array(em), np.array(ee)


@pytest.mark.parametrize("alg", sorted(METHODS))
def test_local_error_orders(alg):
    p, ph = METHODS[alg]
    hs = np.array([0.04, 0.02, 0.01])
    em, ee = local_errors(alg, hs)
    s_main = np.diff(np.log(em)) / np.diff(np.log(hs))
    s_emb = np.diff(np.log(ee)) / np.diff(np.log(hs))
    assert np.all(np.abs(s_main - (p + 1)) < 0.5), s_main
    assert np.all(np.abs(s_emb - (ph + 1)) < 0.5), s_emb


def test_dropped_jacobian_term_is_detected(tmp_path):
    src = oracle.source()
    orig = "r[row] = h * fi[row] + h * Jv;"
    assert src.count(orig) == 1
    with oracle.variant(src.replace(orig, "r[row] = h * fi[row];"), str(tmp_path)):
        hs = np.array([0.04, 0.02, 0.01])
        em, _ = local_errors("rodas5p", hs)
        s_main = np.diff(np.log(em)) / np.diff(np.log(hs))
        assert not np.all(np.abs(s_main - 6) < 0.5)


def rober_f(t, y, k1, k2, k3):
    return [-k1 * y[0] + k3 * y[1] * y[2], k1 * y[0] - k2 * y[1] ** 2 - k3 * y[1] * y[2],
            k2 * y[1] ** 2]


def rober_jac(t, y, k1, k2, k3):
    return [[-k1, k3 * y[2], k3 * y[1]], [k1, -2 * k2 * y[1] - k3 * y[2], -k3 * y[1]],
            [0, 2 * k2 * y[1], 0]]


@pytest.mark.parametrize("alg", sorted(METHODS))
def test_robertson_against_radau(alg):
    import workloads
    P, U, T = workloads.robertson_random(6, seed=3)
    sv = np.logspace(-4, 5, 10)
    out, st, stats = oracle.solve("robertson", alg, P, U, T, abstol=1e-6, reltol=1e-6,
                                  dt0=1e-4, saveat=sv)
    assert np.all(st == 0)
    for i in range(len(P)):
        ref = solve_ivp(rober_f, (0, 1e5), U[i], method="Radau", rtol=1e-12, atol=1e-16,
                        t_eval=sv, jac=rober_jac, args=tuple(P[i])).y.T
        assert np.all(np.abs(out[i] - ref) <= 10 * (1e-6 + 1e-6 * np.abs(ref))), i
    assert np.abs(out.sum(axis=2) - 1).max() < 1e-12
    # f evaluations: the starting f, then s per attempt (stages 2..s and f(y_{n+1}))
    s = len(NODES[alg])
    assert np.all(stats[:, 2] == 1 + s * (stats[:, 0] + stats[:, 1]))
