"""Pins of the oracle's event handling (Sec. 6.5; Appendix, bouncing ball) against the closed
form of the bouncing ball: between impacts the motion is free fall, x(t) = x_k + w_k (t - t_k)
- g (t - t_k)^2 / 2, and each impact turns the arrival speed V into e V upward.  Tsit5 and
its order-4 dense output are exact for this quadratic motion, so the oracle must reproduce
the closed form to rounding: impact count, state at tf, states at save times (dense and
stepped saving), impact times located by the root finder.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def exact(x0, g, e, t):
    """(x, v, impacts before or at t) of a ball dropped at rest from x0."""
    tk, xk, wk, n = 0.0, x0, 0.0, 0
    while True:
        # next impact: xk + wk s - g s^2 / 2 = 0, s > 0
        s = (wk + math.sqrt(wk * wk + 2 * g * xk)) / g
        if tk + s > t:
            d = t - tk
            return xk + wk * d - 0.5 * g * d * d, wk - g * d, n
        tk += s
        V = g * s - wk  # arrival speed (downward)
        wk, xk, n = e * V, 0.0, n + 1


def test_final_state_and_impact_count_match_closed_form():
    P, U, T = workloads.ball(200, seed=3)
    out, st, stats, ev = oracle.solve("ball", "tsit5", P, U, T, abstol=1e-10, reltol=1e-10,
                                      dtmax=1.0, want_events=True)
    assert np.all(st == 0)
    for i in range(len(P)):
        x, v, n = exact(U[i, 0], P[i, 0], P[i, 1], T[i, 1])
        assert ev[i] == n
        assert out[i, 0] == pytest.approx(x, abs=1e-9)
        assert out[i, 1] == pytest.approx(v, abs=1e-9)


@pytest.mark.parametrize("dense", [True, False])
def test_saved_states_match_closed_form(dense):
    P, U, T = workloads.ball(64, seed=4)
    sv = np.linspace(0.0, 15.0, 61)
    out, st, _ = oracle.solve("ball", "tsit5", P, U, T, abstol=1e-10, reltol=1e-10, dtmax=1.0,
                              saveat=sv, dense=dense)
    for i in range(len(P)):
        for k, t in enumerate(sv):
            x, v, _ = exact(U[i, 0], P[i, 0], P[i, 1], t)
            assert out[i, k, 0] == pytest.approx(x, abs=1e-8), (i, t)
            assert out[i, k, 1] == pytest.approx(v, abs=1e-8), (i, t)


def test_impact_times_located_to_rounding():
    """Stop just after each impact: the post-impact velocity is +e V only if the root
    finder put the event before tf; the position shows how far from the true time it is."""
    g, e, x0 = 9.8, 0.8, 50.0
    t1 = math.sqrt(2 * x0 / g)
    for dt_after in (1e-3, 1e-6):
        tf = t1 + dt_after
        out, _, _, ev = oracle.solve("ball", "tsit5", [[g, e]], [[x0, 0.0]], [[0.0, tf]],
                                     abstol=1e-10, reltol=1e-10, dtmax=1.0, want_events=True)
        x, v, n = exact(x0, g, e, tf)
        assert ev[0] == n == 1
        assert out[0, 0] == pytest.approx(x, abs=1e-11)
        assert out[0, 1] == pytest.approx(v, abs=1e-9)


def test_dtmax_caps_steps_and_ball_needs_tsit5():
    P, U, T = workloads.ball(8, seed=5)
    _, _, stats = oracle.solve("ball", "tsit5", P, U, T, abstol=1e-8, reltol=1e-8, dtmax=0.5)
    assert np.all(stats[:, 0] >= 30)
    for alg, kw in (("rk4", dict(dt=0.01)), ("ros23", {})):
        with pytest.raises(ValueError):
            oracle.solve("ball", alg, P, U, T, **kw)


def test_without_dtmax_large_steps_still_find_every_impact():
    """Error estimates are ~0 for free fall, so steps grow 10x per step; the 10 checkpoints
    per step must still catch every impact while flights are long compared with h/10."""
    P, U, T = workloads.ball(32, seed=6, t1=8.0)
    out, _, _, ev = oracle.solve("ball", "tsit5", P, U, T, abstol=1e-10, reltol=1e-10,
                                 want_events=True)
    for i in range(len(P)):
        x, v, n = exact(U[i, 0], P[i, 0], P[i, 1], T[i, 1])
        assert ev[i] == n and out[i, 0] == pytest.approx(x, abs=1e-8)
