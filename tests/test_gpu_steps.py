"""GPU parity of the every-step record (ens_opts.step_cap: the full solution of adaptive
solves) against the oracle's record, through the C ABI.

* FP64 Lorenz: equal counts (accepted steps + 1) on >= 99 % of trajectories, step times
  within 1e-5 of the oracle's (the kernels' step-size controller forms its ratio and factor
  in FP32 in both precisions, so FP64 step sizes agree with the oracle's to float precision),
  and every recorded step is the method's step: the oracle's FP64 Tsit5 step from each
  recorded (t_k, u_k) with h = t_{k+1} - t_k reproduces u_{k+1} to 1e-12.  The last entry is
  the plain solve's final state, bit for bit.  SoA equals row-major bit for bit.
* The record does not change the solve: its last entry equals the final state of the same
  solve without a record, bit for bit (FP32, one trajectory per thread).
* A small capacity keeps the first entries and reports the full count.
* Events: the bouncing ball's record has the oracle's counts and its impacts (the entries at
  x = 0, with the post-affect velocities); its step times differ early on, as its error
  estimate is rounding noise that the FP32 and FP64 controllers turn into different growth.
* step_cap with save times or with a fixed-step method is rejected.
"""
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


@pytest.fixture(scope="module")
def lor():
    from paper_2304_06835_gb300 import EnsembleSolver
    s = EnsembleSolver("lorenz")
    yield s
    s.close()


def test_record_fp64_matches_oracle_and_soa(lor):
    P, U, T = workloads.lorenz_random(1000 + 21, seed=51, t1=1.0)
    cap, kw = 192, dict(abstol=1e-8, reltol=1e-8)
    rt, ru, rn, _, _, _ = oracle.solve_steps("lorenz", "tsit5", P, U, T, cap, **kw)
    t, u, n, st, _ = lor.solve_steps(dev(P), dev(U), dev(T), cap, **kw)
    t, u, n = host(t), host(u), n.cpu().numpy()
    assert int(st.abs().sum()) == 0 and np.all(rn <= cap)
    eq = n == rn
    assert eq.mean() >= 0.99
    for i in np.flatnonzero(eq):
        np.testing.assert_allclose(t[i, :n[i]], rt[i, :n[i]], rtol=1e-5, atol=1e-12)
    for i in range(0, len(P), 97):  # replay every step of a sample through the oracle
        for j in range(n[i] - 1):
            nxt, _ = oracle.step("lorenz", "tsit5", u[i, j], P[i], t[i, j], t[i, j + 1] - t[i, j])
            assert np.abs(nxt - u[i, j + 1]).max() <= 1e-12 * max(np.abs(nxt).max(), 1.0)
    f, _, _ = lor.solve(dev(P), dev(U), dev(T), alg="tsit5", **kw)
    np.testing.assert_array_equal(u[np.arange(len(P)), n - 1], host(f))
    s = lambda a: dev(np.ascontiguousarray(a.T))
    t2, u2, n2, _, _ = lor.solve_steps(s(P), s(U), s(T), cap, layout="soa", **kw)
    np.testing.assert_array_equal(n2.cpu().numpy(), n)
    np.testing.assert_array_equal(np.transpose(host(u2), (2, 0, 1)), u)
    np.testing.assert_array_equal(host(t2).T, t)


def test_record_leaves_the_solve_unchanged_fp32(lor):
    P, U, T = workloads.lorenz_random(4096, seed=52, t1=2.0)
    f = lambda a: dev(a, torch.float32)
    kw = dict(abstol=1e-5, reltol=1e-5, schedule="persistent", tpt=1)
    t, u, n, _, stats = lor.solve_steps(f(P), f(U), f(T), 512, want_stats=True, **kw)
    out, _, fstats = lor.solve(f(P), f(U), f(T), alg="tsit5", want_stats=True, **kw)
    n = n.cpu().numpy()
    np.testing.assert_array_equal(fstats.cpu().numpy(), stats.cpu().numpy())
    assert np.all(n == stats.cpu().numpy()[0] + 1) and np.all(n <= 512)
    np.testing.assert_array_equal(host(u)[np.arange(4096), n - 1], host(out))
    np.testing.assert_array_equal(host(t)[np.arange(4096), n - 1], T[:, 1].astype(np.float32))


def test_small_capacity_keeps_first_entries(lor):
    P, U, T = workloads.lorenz_random(500, seed=53, t1=1.0)
    kw = dict(abstol=1e-8, reltol=1e-8)
    ta, ua, na, _, _ = lor.solve_steps(dev(P), dev(U), dev(T), 256, **kw)
    tb, ub, nb, _, _ = lor.solve_steps(dev(P), dev(U), dev(T), 7, **kw)
    np.testing.assert_array_equal(na.cpu().numpy(), nb.cpu().numpy())
    assert np.all(nb.cpu().numpy() > 7)
    np.testing.assert_array_equal(host(ua)[:, :7], host(ub))
    np.testing.assert_array_equal(host(ta)[:, :7], host(tb))


def test_record_with_events_matches_oracle():
    from paper_2304_06835_gb300 import EnsembleSolver
    b = EnsembleSolver("ball")
    P, U, T = workloads.ball(300, seed=54)
    cap, kw = 128, dict(abstol=1e-10, reltol=1e-10, dtmax=1.0)
    rt, ru, rn, _, _, _ = oracle.solve_steps("ball", "tsit5", P, U, T, cap, **kw)
    t, u, n, _, _ = b.solve_steps(dev(P), dev(U), dev(T), cap, **kw)
    t, u, n = host(t), host(u), n.cpu().numpy()
    np.testing.assert_array_equal(n, rn)
    for i in range(300):
        k = n[i]
        # free fall is integrated exactly, so the error estimate is rounding noise and the
        # FP32-formed step factor grows the first steps differently from the oracle's FP64
        # one: compare the impacts (entries at x = 0), not the step times
        ground = np.abs(u[i, :k, 0]) < 1e-9
        np.testing.assert_array_equal(ground, np.abs(ru[i, :k, 0]) < 1e-9)
        np.testing.assert_allclose(u[i, :k, 1][ground], ru[i, :k, 1][ground], rtol=1e-9)
    b.close()


def test_step_cap_rejections(lor):
    import ctypes

    from paper_2304_06835_gb300 import EnsError, _lib, make_opts
    P, U, T = workloads.lorenz_random(8, seed=55, t1=1.0)
    with pytest.raises(EnsError):
        lor.solve_steps(dev(P), dev(U), dev(T), 16, alg="tsit5_fixed")
    Pd, Ud, Td = dev(P), dev(U), dev(T)
    n = torch.empty(8, dtype=torch.int32, device="cuda")
    out = torch.empty((8, 16, 3), dtype=torch.float64, device="cuda")
    opts, keep = make_opts("tsit5", _lib.F64, "rowmajor", 0.0, 1e-6, 1e-6, saveat=[0.5],
                           step_cap=16, step_n=n)
    ptr = lambda x: ctypes.c_void_p(x.data_ptr())
    with pytest.raises(EnsError):  # save times and a step record together
        _lib.check(_lib.lib().ens_solve(lor._h, 8, ptr(Pd), ptr(Ud), ptr(Td), ctypes.byref(opts),
                                        ptr(out), None, None, None))
    del keep
