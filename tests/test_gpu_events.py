"""GPU parity of event handling (the bouncing ball, Sec. 6.5) and of the adaptive step cap
dtmax, through the C ABI, against the oracle and the closed form.

* FP64: final states and saved states (dense and stepped saving) within 1e-12 of the
  oracle, which runs the same detection and root finding; step counts identical; the
  GPU's states within 1e-8 of the closed form.
* FP32: within 2e-3 of the closed form (event times are located to 4 float ulp of a step).
* Launch shapes (direct, persistent one or two trajectories per thread) give bit-identical
  results; the ball accepts only adaptive Tsit5.
* dtmax: Lorenz with a step cap against the oracle's capped solve (1e-12, same counts);
  two trajectories per thread with dtmax (the generic kernel) equal one per thread.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def dev(a, dt=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().double().numpy()


def exact(x0, g, e, t):
    tk, xk, wk = 0.0, x0, 0.0
    while True:
        s = (wk + math.sqrt(wk * wk + 2 * g * xk)) / g
        if tk + s > t:
            d = t - tk
            return xk + wk * d - 0.5 * g * d * d, wk - g * d
        tk += s
        wk, xk = e * (g * s - wk), 0.0


@pytest.fixture(scope="module")
def ball():
    from paper_2304_06835_gb300 import EnsembleSolver
    s = EnsembleSolver("ball")
    yield s
    s.close()


KW = dict(abstol=1e-10, reltol=1e-10, dtmax=1.0)


@pytest.mark.parametrize("schedule,tpt", [("direct", 0), ("persistent", 1), ("persistent", 2)])
def test_ball_fp64_matches_oracle_and_closed_form(ball, schedule, tpt):
    P, U, T = workloads.ball(1000 + 29, seed=41)
    ref, rst, rstats = oracle.solve("ball", "tsit5", P, U, T, **KW)
    out, st, stats = ball.solve(dev(P), dev(U), dev(T), alg="tsit5", schedule=schedule, tpt=tpt,
                                want_stats=True, **KW)
    o = host(out)
    assert int(st.abs().sum()) == 0
    np.testing.assert_array_equal(stats.cpu().numpy().T[:, :2], rstats[:, :2])
    assert np.abs(o - ref).max() <= 1e-12 * 50
    for i in range(0, len(P), 37):
        x, v = exact(U[i, 0], P[i, 0], P[i, 1], T[i, 1])
        assert abs(o[i, 0] - x) <= 1e-8 and abs(o[i, 1] - v) <= 1e-8


def test_ball_launch_shapes_bit_identical(ball):
    P, U, T = workloads.ball(4096, seed=42)
    outs = [host(ball.solve(dev(P), dev(U), dev(T), alg="tsit5", schedule=s, tpt=t, **KW)[0])
            for s, t in (("direct", 0), ("persistent", 1), ("persistent", 2))]
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


@pytest.mark.parametrize("dense", [True, False])
def test_ball_saves_fp64(ball, dense):
    P, U, T = workloads.ball(300, seed=43)
    sv = np.linspace(0.0, 15.0, 31)
    ref, _, _ = oracle.solve("ball", "tsit5", P, U, T, saveat=sv, dense=dense, **KW)
    out, _, _ = ball.solve(dev(P), dev(U), dev(T), alg="tsit5", saveat=sv, dense=dense, **KW)
    o = host(out)
    assert np.abs(o - ref).max() <= 1e-12 * 50
    for i in range(0, 300, 29):
        for k in (3, 17, 30):
            x, v = exact(U[i, 0], P[i, 0], P[i, 1], sv[k])
            assert abs(o[i, k, 0] - x) <= 1e-8 and abs(o[i, k, 1] - v) <= 1e-8


def test_ball_fp32_close_to_closed_form(ball):
    P, U, T = workloads.ball(8192, seed=44)
    f = lambda a: dev(a, torch.float32)
    out, st, _ = ball.solve(f(P), f(U), f(T), alg="tsit5", abstol=1e-6, reltol=1e-6, dtmax=1.0)
    o = host(out)
    assert int(st.abs().sum()) == 0
    P32 = np.asarray(P, np.float32).astype(np.float64)
    err = max(max(abs(o[i, 0] - x), abs(o[i, 1] - v))
              for i in range(0, 8192, 61)
              for x, v in [exact(50.0, P32[i, 0], P32[i, 1], 15.0)])
    assert err <= 2e-3, err


def test_ball_rejects_other_methods(ball):
    from paper_2304_06835_gb300 import EnsError
    P, U, T = workloads.ball(4, seed=45)
    for alg, kw in (("rk4", dict(dt=0.01)), ("tsit5_fixed", dict(dt=0.01)), ("ros23", {})):
        with pytest.raises(EnsError):
            ball.solve(dev(P), dev(U), dev(T), alg=alg, **kw)


def test_dtmax_lorenz_matches_oracle_and_skips_the_pair_kernel():
    from paper_2304_06835_gb300 import EnsembleSolver
    s = EnsembleSolver("lorenz")
    P, U, T = workloads.lorenz_random(1024, seed=46, t1=1.0)
    kw = dict(abstol=1e-8, reltol=1e-8, dtmax=0.01)
    ref, _, rstats = oracle.solve("lorenz", "tsit5", P, U, T, **kw)
    out, _, stats = s.solve(dev(P), dev(U), dev(T), alg="tsit5", want_stats=True, **kw)
    g = stats.cpu().numpy().T
    assert np.all(g[:, 0] >= 100)
    same = np.all(g[:, :2] == rstats[:, :2], axis=1)
    assert same.mean() >= 0.99
    o = host(out)
    rel = np.abs(o - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1)
    assert rel[same].max() <= 1e-12
    f = lambda a: dev(a, torch.float32)
    a1 = host(s.solve(f(P), f(U), f(T), alg="tsit5", schedule="persistent", tpt=1,
                      abstol=1e-5, reltol=1e-5, dtmax=0.01)[0])
    a2 = host(s.solve(f(P), f(U), f(T), alg="tsit5", schedule="persistent", tpt=2,
                      abstol=1e-5, reltol=1e-5, dtmax=0.01)[0])
    np.testing.assert_array_equal(a1, a2)
    s.close()
