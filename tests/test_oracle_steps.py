"""Pins of the oracle's every-step record of adaptive solves (the full-trajectory output):

* entry 0 is (t0, u0), the last entry is (tf, final state), the times increase strictly and
  the count is accepted steps + 1;
* replay: one Tsit5 step from each recorded (t_k, u_k) with h = t_{k+1} - t_k reproduces
  u_{k+1} -- the record is the method's own step sequence (no interpolation, nothing skipped);
* a capacity smaller than the step count keeps the first entries and reports the full count;
* with events the record holds the post-event states at the event times.
"""
import numpy as np

import oracle
import workloads


def test_record_structure_and_replay():
    P, U, T = workloads.lorenz_random(16, seed=3, t1=1.0)
    t, u, n, out, st, stats = oracle.solve_steps("lorenz", "tsit5", P, U, T, 256, abstol=1e-7,
                                                 reltol=1e-7)
    assert np.all(st == 0) and np.all(n == stats[:, 0] + 1) and np.all(n <= 256)
    for i in range(16):
        k = n[i]
        assert t[i, 0] == T[i, 0] and t[i, k - 1] == T[i, 1]
        np.testing.assert_array_equal(u[i, 0], U[i])
        np.testing.assert_array_equal(u[i, k - 1], out[i])
        assert np.all(np.diff(t[i, :k]) > 0) and np.all(np.isnan(t[i, k:]))
        for j in range(k - 1):
            nxt, _ = oracle.step("lorenz", "tsit5", u[i, j], P[i], t[i, j], t[i, j + 1] - t[i, j])
            np.testing.assert_allclose(nxt, u[i, j + 1], rtol=1e-13, atol=1e-13)


def test_capacity_keeps_the_first_entries():
    P, U, T = workloads.lorenz_random(8, seed=4, t1=1.0)
    full = oracle.solve_steps("lorenz", "tsit5", P, U, T, 512, abstol=1e-8, reltol=1e-8)
    part = oracle.solve_steps("lorenz", "tsit5", P, U, T, 10, abstol=1e-8, reltol=1e-8)
    assert np.all(part[2] == full[2]) and np.all(full[2] > 10)
    np.testing.assert_array_equal(part[0], full[0][:, :10])
    np.testing.assert_array_equal(part[1], full[1][:, :10])


def test_events_appear_in_the_record():
    P, U, T = workloads.ball(8, seed=5)
    t, u, n, out, st, _ = oracle.solve_steps("ball", "tsit5", P, U, T, 512, abstol=1e-10,
                                             reltol=1e-10, dtmax=1.0)
    for i in range(8):
        k = n[i]
        ground = np.flatnonzero(np.abs(u[i, :k, 0]) < 1e-9)
        assert len(ground) >= 2  # at least two impacts in [0, 15] for e >= 0.7
        assert np.all(u[i, ground, 1] > 0)  # post-affect: moving up
        # the first impact time is the free-fall time from x0
        assert abs(t[i, ground[0]] - np.sqrt(2 * U[i, 0] / P[i, 0])) < 1e-9
