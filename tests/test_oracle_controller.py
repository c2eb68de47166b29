"""Pins of the oracle's step-size controller and starting step (CPU only).

The PI controller of Sec. 3.1 sets h_new = eta * q_n^(-beta1) * q_(n-1)^(beta2) * h after an
accepted step (beta1, beta2 > 0 in this sign convention).  On u' = lam*u with lam < 0 and a
purely relative tolerance, the scaled error ratio q of a step of size h does not depend on
the state (E and the scale are both proportional to |u_n|), so q is a function of h alone.
If the controller settles, consecutive ratios are equal and the accepted steps are constant,
which forces eta * q^(beta2 - beta1) = 1, i.e.

    q* = eta^(1 / (beta1 - beta2))

whatever the method's error function is: 0.9^(1/0.06) = 0.17273 for Tsit5 (beta1 = 0.7/5,
beta2 = 0.4/5) and 0.9^(1/0.1) = 0.34868 for Rosenbrock23 (0.7/3, 0.4/3).  A flipped sign of
beta2 moves the fixed point to eta^(1/(beta1 + beta2)) (0.619 for Tsit5), swapped exponents
make the loop unstable, a controller that never updates q_(n-1) settles elsewhere, and an
inverted clamp pins the factor at a bound: `test_controller_mutations_are_detected` plants
each of these in a copy of the oracle and checks that the fixed-point pin fails.

The starting step is Hairer-Norsett-Wanner I, II.4 (the paper gives only Robertson's fixed
h0 = 1e-4).  On u' = lam*u from u0 with sc = atol + rtol*|u0| the algorithm reduces by hand to

    d0 = |u0|/sc,  d1 = |lam u0|/sc,  h0 = 0.01 d0/d1 = 0.01/|lam|   (1e-6 if d0 or d1 < 1e-5)
    d2 = |f(u0 + h0 f0) - f0| / (sc h0) = lam^2 |u0| / sc
    h1 = (0.01 / max(d1, d2))^(1/(p+1))       (max(1e-6, 1e-3 h0) if max(d1, d2) <= 1e-15)
    h  = min(100 h0, h1)

with p the method's order (5 for Tsit5, 2 for Rosenbrock23).  The first accepted step of the
oracle's solve must equal that h.
"""
import math

import numpy as np
import pytest

import oracle

ETA = 0.9
Q_STAR = {"tsit5": ETA ** (1.0 / (0.7 / 5 - 0.4 / 5)), "ros23": ETA ** (1.0 / (0.7 / 3 - 0.4 / 3))}


def _steady_ratio(alg, lam, rtol, span):
    """Run u' = lam*u (the GBM drift with no noise) adaptively; return the accepted steps'
    relative spread over the last 20 steps and the error ratio q at the settled step."""
    P = np.array([[lam, 0.0]])
    U = np.array([[1.0]])
    T = np.array([[0.0, span]])
    rt, _, rn, _, st, _ = oracle.solve_steps("gbm", alg, P, U, T, 20000, abstol=1e-300,
                                             reltol=rtol)
    assert st[0] == 0
    n = int(rn[0])
    assert n <= 20000
    h = np.diff(rt[0, :n])[:-1]  # the last step is clamped onto tf
    tail = h[-20:]
    spread = (tail.max() - tail.min()) / tail.mean()
    hs = float(tail[-1])
    un, err = oracle.step("gbm", alg, [1.0], [lam, 0.0], 0.0, hs)
    # scale = atol + rtol * max(|u_n|, |u_n+1|) with u_n = 1 and a decaying solution
    q = abs(err[0]) / (rtol * max(1.0, abs(un[0])))
    return spread, q


def _fixed_point_holds(alg, lam, rtol, span):
    # E ~ q* rtol |u| is a difference of O(|u|) stage sums, so it carries a relative
    # round-off of ~1e-16 / rtol; at rtol >= 1e-7 that leaves q and the steps settled to 1e-7
    spread, q = _steady_ratio(alg, lam, rtol, span)
    return spread < 1e-7 and abs(q / Q_STAR[alg] - 1.0) < 1e-6, (spread, q)


CASES = [("tsit5", -1.0, 1e-6, 40.0), ("tsit5", -3.0, 1e-7, 20.0),
         ("ros23", -1.0, 1e-6, 40.0), ("ros23", -0.2, 1e-4, 400.0)]


@pytest.mark.parametrize("alg,lam,rtol,span", CASES)
def test_pi_controller_fixed_point(alg, lam, rtol, span):
    ok, (spread, q) = _fixed_point_holds(alg, lam, rtol, span)
    assert ok, (spread, q, Q_STAR[alg])


# Each entry: (exact text in the oracle's accept branch, planted replacement, what it models).
CONTROLLER_MUTATIONS = [
    ("std::pow(qg, -beta1) * std::pow(qold, beta2)",
     "std::pow(qg, -beta1) * std::pow(qold, -beta2)", "beta2 sign flipped"),
    ("std::pow(qg, -beta1) * std::pow(qold, beta2)",
     "std::pow(qg, -beta2) * std::pow(qold, beta1)", "exponents swapped"),
    ("qold = std::max(q, T(QOLD_INIT));", "qold = T(QOLD_INIT);", "q_(n-1) never updated"),
    ("fac = std::min(T(FAC_MAX), std::max(T(FAC_MIN), fac));",
     "fac = std::max(T(FAC_MAX), std::min(T(FAC_MIN), fac));", "clamp inverted"),
]


@pytest.mark.parametrize("orig,planted,what", CONTROLLER_MUTATIONS,
                         ids=[m[2] for m in CONTROLLER_MUTATIONS])
def test_controller_mutations_are_detected(tmp_path, orig, planted, what):
    src = oracle.source()
    assert src.count(orig) == 1, "the oracle's controller text changed: update the mutation"
    with oracle.variant(src.replace(orig, planted), str(tmp_path)):
        for alg, lam, rtol, span in (CASES[0], CASES[2]):
            try:
                ok, _ = _fixed_point_holds(alg, lam, rtol, span)
            except AssertionError:  # the planted controller failed the solve or ran away
                ok = False
            assert not ok, "planted mistake not detected: " + what


def hnw_closed_form(lam, u0, atol, rtol, order):
    sc = atol + rtol * abs(u0)
    d0 = abs(u0) / sc
    d1 = abs(lam * u0) / sc
    h0 = 1e-6 if (d0 < 1e-5 or d1 < 1e-5) else 0.01 / abs(lam)
    d2 = lam * lam * abs(u0) / sc
    dm = max(d1, d2)
    h1 = max(1e-6, 1e-3 * h0) if dm <= 1e-15 else (0.01 / dm) ** (1.0 / (order + 1))
    return min(100 * h0, h1)


# (lam, u0, atol, rtol): |lam| < 1 (d1 > d2), |lam| > 1, the 100 h0 bound active,
# d0 < 1e-5 (tiny state), lam = 0 (d1 = d2 = 0)
START_CASES = [(-0.5, 1.0, 1e-8, 1e-6), (-3.0, 2.0, 1e-6, 1e-3), (-40.0, 1.0, 1e-3, 1e-3),
               (2.0, 5.0, 1e-10, 1e-8), (-1.0, 1e-8, 1e-2, 1e-6), (0.0, 1.0, 1e-6, 1e-6)]


def _first_step(alg, lam, u0, atol, rtol):
    P = np.array([[lam, 0.0]])
    U = np.array([[u0]])
    T = np.array([[0.0, 1e3]])
    rt, _, rn, _, _, _ = oracle.solve_steps("gbm", alg, P, U, T, 4, abstol=atol, reltol=rtol,
                                            maxiters=3)
    return rt[0, 1] - rt[0, 0]


@pytest.mark.parametrize("alg,order", [("tsit5", 5), ("ros23", 2)])
@pytest.mark.parametrize("lam,u0,atol,rtol", START_CASES)
def test_starting_step_closed_form(alg, order, lam, u0, atol, rtol):
    h = _first_step(alg, lam, u0, atol, rtol)
    ref = hnw_closed_form(lam, u0, atol, rtol, order)
    assert math.isclose(h, ref, rel_tol=1e-13), (h, ref)


START_MUTATIONS = [
    ("std::pow(T(0.01) / dm, T(1.0 / (order + 1)))", "std::pow(T(0.01) / dm, T(1.0 / order))",
     "exponent 1/p"),
    ("T dm = std::max(d1, d2);", "T dm = d2;", "d1 dropped from the maximum"),
    ("return std::min(T(100) * h0, h1);", "return h1;", "100 h0 bound dropped"),
    ("T(0.01) * d0 / d1;", "T(0.01) * d1 / d0;", "h0 ratio inverted"),
]


@pytest.mark.parametrize("orig,planted,what", START_MUTATIONS, ids=[m[2] for m in START_MUTATIONS])
def test_starting_step_mutations_are_detected(tmp_path, orig, planted, what):
    src = oracle.source()
    assert src.count(orig) == 1, "the oracle's starting-step text changed: update the mutation"
    with oracle.variant(src.replace(orig, planted), str(tmp_path)):
        bad = 0
        for lam, u0, atol, rtol in START_CASES:
            h = _first_step("tsit5", lam, u0, atol, rtol)
            bad += not math.isclose(h, hnw_closed_form(lam, u0, atol, rtol, 5), rel_tol=1e-13)
        assert bad > 0, "planted mistake not detected: " + what
