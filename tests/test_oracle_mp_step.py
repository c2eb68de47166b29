"""Single steps of the oracle against the same step evaluated in 50-digit arithmetic (mpmath).

Each method's step is written out here from its published form, independently of the
oracle's C++: Rosenbrock23 from Shampine and Reichelt's ode23s scheme (d = 1/(2 + sqrt 2),
e32 = 6 + sqrt 2, W = I - h d J; Sec. 5.2.1 names the method), Rodas4 / Rodas5P from the
standard Rosenbrock form of Hairer and Wanner II, IV.7 (W k_i = h f(y + sum alpha_ij k_j)
+ h J sum gamma_ij k_j with W = I - h gamma J) on the coefficients the oracle holds (pinned
by the order conditions in test_oracle_rodas.py), Tsit5 from its Butcher tableau (pinned in
test_oracle_tableau.py).  The models are the Appendix's Robertson and Lorenz equations with
their Jacobians taken by hand.  Steps on stiff Robertson states (h J up to 10^5) and on
Lorenz: the FP64 oracle agrees to 1e-12 relative in the new state (what FP64 rounding of a
well-conditioned step allows) and the error estimates to 1e-9 of their size plus 1e-14 of
the state's (the estimate is a difference at the state's scale); a mistaken coefficient or
stage term in either implementation is orders of magnitude larger.
"""
import mpmath as mp
import numpy as np
import pytest

import oracle

mp.mp.dps = 50


def rob_f(u, p):
    k1, k2, k3 = p
    y1, y2, y3 = u
    return [-k1 * y1 + k3 * y2 * y3, k1 * y1 - k2 * y2 * y2 - k3 * y2 * y3, k2 * y2 * y2]


def rob_J(u, p):
    k1, k2, k3 = p
    y1, y2, y3 = u
    return mp.matrix([[-k1, k3 * y3, k3 * y2],
                      [k1, -2 * k2 * y2 - k3 * y3, -k3 * y2],
                      [0, 2 * k2 * y2, 0]])


def lor_f(u, p):
    s, r, b = p
    x, y, z = u
    return [s * (y - x), x * (r - z) - y, x * y - b * z]


def lor_J(u, p):
    s, r, b = p
    x, y, z = u
    return mp.matrix([[-s, s, 0], [r - z, -1, -x], [y, x, -b]])


def vec(a):
    return mp.matrix([mp.mpf(float(x)) for x in a])


def mp_ros23(f, J, u, p, h):
    d = 1 / (2 + mp.sqrt(2))
    e32 = 6 + mp.sqrt(2)
    u, h = vec(u), mp.mpf(h)
    p = [mp.mpf(float(x)) for x in p]
    W = mp.eye(3) - h * d * J(u, p)
    f0 = mp.matrix(f(u, p))
    k1 = mp.lu_solve(W, f0)
    f1 = mp.matrix(f(u + h / 2 * k1, p))
    k2 = mp.lu_solve(W, f1 - k1) + k1
    un = u + h * k2
    f2 = mp.matrix(f(un, p))
    k3 = mp.lu_solve(W, f2 - e32 * (k2 - f1) - 2 * (k1 - f0))
    return un, h / 6 * (k1 - 2 * k2 + k3)


def mp_rodas(f, J, u, p, h, tab):
    gamma, alpha, G, b, bh = tab
    s = len(b)
    u, h = vec(u), mp.mpf(h)
    p = [mp.mpf(float(x)) for x in p]
    Ju = J(u, p)
    W = mp.eye(3) - h * mp.mpf(gamma) * Ju
    k = []
    for i in range(s):
        arg = u + sum((mp.mpf(alpha[i, j]) * k[j] for j in range(i)), mp.matrix(3, 1))
        gsum = sum((mp.mpf(G[i, j]) * k[j] for j in range(i)), mp.matrix(3, 1))
        k.append(mp.lu_solve(W, h * mp.matrix(f(arg, p)) + h * (Ju * gsum)))
    un = u + sum((mp.mpf(b[j]) * k[j] for j in range(s)), mp.matrix(3, 1))
    uh = u + sum((mp.mpf(bh[j]) * k[j] for j in range(s)), mp.matrix(3, 1))
    return un, un - uh


def mp_tsit5(f, u, p, h):
    c, A, b, bh = oracle.tsit5_tableau()
    u, h = vec(u), mp.mpf(h)
    p = [mp.mpf(float(x)) for x in p]
    k = []
    for i in range(7):
        arg = u + h * sum((mp.mpf(A[i, j]) * k[j] for j in range(i)), mp.matrix(3, 1))
        k.append(mp.matrix(f(arg, p)))
    un = u + h * sum((mp.mpf(b[j]) * k[j] for j in range(7)), mp.matrix(3, 1))
    # the embedded solution minus the step's (only |E| enters the error norm)
    e = h * sum((mp.mpf(bh[j] - b[j]) * k[j] for j in range(7)), mp.matrix(3, 1))
    return un, e


ROB_P = [0.04, 3e7, 1e4]
ROB_STATES = [[1 - 1e-4, 3.0e-5, 7.0e-5], [0.8, 1.2e-5, 0.2], [0.02, 8.0e-8, 0.98]]
LOR_P = [10.0, 28.0, 8.0 / 3.0]
LOR_STATES = [[1.0, 0.0, 0.0], [-8.5, -7.1, 29.4], [12.0, 15.0, 20.0]]


def check(un_o, e_o, un_m, e_m):
    un_m = np.array([float(x) for x in un_m])
    e_m = np.array([float(x) for x in e_m])
    du = np.abs(un_o - un_m).max() / np.abs(un_m).max()
    de = np.abs(e_o - e_m).max() / (np.abs(e_m).max() + 1e-16)
    assert du <= 1e-12, du
    # the estimate is a difference of stage sums at the scale of the state: its FP64 rounding
    # is absolute, ~1e-16 of |u|
    assert np.all(np.abs(e_o - e_m) <= 1e-9 * np.abs(e_m).max() + 1e-14 * np.abs(un_m).max()), de
    return du, de


@pytest.mark.parametrize("h", [1e-4, 1e-2, 1.0, 100.0])
@pytest.mark.parametrize("u", ROB_STATES)
def test_rosenbrock23_step_50_digits(u, h):
    un, e = oracle.step("robertson", "ros23", u, ROB_P, 0.0, h)
    check(un, e, *mp_ros23(rob_f, rob_J, u, ROB_P, h))


@pytest.mark.parametrize("alg", ["rodas4", "rodas5p"])
@pytest.mark.parametrize("h", [1e-3, 1.0, 100.0])
@pytest.mark.parametrize("u", ROB_STATES)
def test_rodas_step_50_digits(alg, u, h):
    un, e = oracle.step("robertson", alg, u, ROB_P, 0.0, h)
    check(un, e, *mp_rodas(rob_f, rob_J, u, ROB_P, h, oracle.rosenbrock_tableau(alg)))


@pytest.mark.parametrize("h", [1e-3, 1e-2])
@pytest.mark.parametrize("u", LOR_STATES)
def test_lorenz_steps_50_digits(u, h):
    un, e = oracle.step("lorenz", "tsit5", u, LOR_P, 0.0, h)
    check(un, e, *mp_tsit5(lor_f, u, LOR_P, h))
    un, e = oracle.step("lorenz", "ros23", u, LOR_P, 0.0, h)
    check(un, e, *mp_ros23(lor_f, lor_J, u, LOR_P, h))
