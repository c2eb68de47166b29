"""GPU parity of the dense output (adaptive Tsit5 with dense=True) against the oracle's dense
saving on the same inputs, through the C ABI.

* FP64, non-chaotic Lorenz (rho < 10, [0, 10]) and the [0, 1] workload: every save within
  1e-12 of the oracle (normwise, both follow the same steps and the same interpolant);
  identical step counts.
* The steps and the final state equal those of the same GPU solve without save times,
  bit for bit (dense saving does not touch the step sequence).
* Save times before t0 / after tf are NaN, at t0 / tf the initial / final state.
* FP32: every save within 10x tolerance of a tol-1e-12 FP64 reference.
* Rosenbrock23 ignores the flag (bit-identical to the stepped saving).
* Dense saves equal across the direct and persistent schedules, bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

SV = np.array([-1.0, 0.0, 0.0137, 0.25, 0.5, 0.75, 0.999, 1.0, 2.0])


def dev(a, dt=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().double().numpy()


def normwise(out, ref):
    d = np.abs(out - ref)
    return np.nanmax(d.reshape(d.shape[0], -1), axis=1) / np.maximum(
        np.nanmax(np.abs(ref).reshape(ref.shape[0], -1), axis=1), 1.0)


@pytest.fixture(scope="module")
def lor():
    from paper_2304_06835_gb300 import EnsembleSolver
    s = EnsembleSolver("lorenz")
    yield s
    s.close()


def _nonchaotic(N, t1):
    P, U, T = workloads.lorenz_random(N, seed=31, t1=t1)
    P[:, 1] = np.linspace(0.5, 9.5, N)
    return P, U, T


@pytest.mark.parametrize("schedule", ["direct", "persistent"])
@pytest.mark.parametrize("t1", [1.0, 10.0])
def test_dense_fp64_matches_oracle(lor, schedule, t1):
    N = 700 + 13
    P, U, T = _nonchaotic(N, t1) if t1 > 1 else workloads.lorenz_random(N, seed=32, t1=t1)
    sv = SV * t1
    kw = dict(abstol=1e-8, reltol=1e-8)
    ref, rst, rstats = oracle.solve("lorenz", "tsit5", P, U, T, saveat=sv, dense=True, **kw)
    out, st, stats = lor.solve(dev(P), dev(U), dev(T), alg="tsit5", saveat=sv, dense=True,
                               schedule=schedule, want_stats=True, **kw)
    o = host(out)
    np.testing.assert_array_equal(np.isnan(o), np.isnan(ref))
    assert np.all(np.isnan(o[:, 0])) and np.all(np.isnan(o[:, -1]))
    np.testing.assert_array_equal(o[:, 1], U)
    g = stats.cpu().numpy().T
    same = np.all(g[:, :2] == rstats[:, :2], axis=1)
    assert same.mean() >= 0.99
    assert normwise(o[same], ref[same]).max() <= 1e-12
    # the steps and the final state are those of the solve without save times
    f, _, fstats = lor.solve(dev(P), dev(U), dev(T), alg="tsit5", schedule=schedule,
                             want_stats=True, **kw)
    np.testing.assert_array_equal(fstats.cpu().numpy(), stats.cpu().numpy())
    np.testing.assert_array_equal(host(f), o[:, 7])


def test_dense_soa_layout_equals_rowmajor(lor):
    P, U, T = workloads.lorenz_random(1000, seed=33, t1=1.0)
    kw = dict(abstol=1e-7, reltol=1e-7, saveat=SV, dense=True)
    o1, _, _ = lor.solve(dev(P), dev(U), dev(T), alg="tsit5", **kw)
    t = lambda a: dev(np.ascontiguousarray(a.T))
    o2, _, _ = lor.solve(t(P), t(U), t(T), alg="tsit5", layout="soa", **kw)
    np.testing.assert_array_equal(host(o1), np.transpose(host(o2), (2, 0, 1)))


def test_dense_fp32_within_tolerance_of_reference(lor):
    P, U, T = _nonchaotic(2048, 10.0)
    P, U, T = (np.asarray(a, np.float32).astype(np.float64) for a in (P, U, T))
    sv = SV * 10.0
    tol = 1e-5
    ref, _, _ = oracle.solve("lorenz", "tsit5", P, U, T, abstol=1e-12, reltol=1e-12, saveat=sv)
    d32 = lambda a: dev(a, torch.float32)
    out, st, _ = lor.solve(d32(P), d32(U), d32(T), alg="tsit5", abstol=tol, reltol=tol,
                           saveat=sv, dense=True)
    o = host(out)
    assert int(st.abs().sum()) == 0
    inner = (slice(None), slice(1, 8))
    assert np.all(np.abs(o[inner] - ref[inner]) <= 10 * (tol + tol * np.abs(ref[inner])))


def test_dense_flag_ignored_by_rosenbrock():
    from paper_2304_06835_gb300 import EnsembleSolver
    r = EnsembleSolver("robertson")
    P, U, T = workloads.robertson_random(256, seed=34, t1=100.0)
    sv = [0.0, 1.0, 10.0, 100.0]
    kw = dict(abstol=1e-6, reltol=1e-6, dt0=1e-4, saveat=sv)
    a, _, _ = r.solve(dev(P), dev(U), dev(T), alg="ros23", dense=True, **kw)
    b, _, _ = r.solve(dev(P), dev(U), dev(T), alg="ros23", **kw)
    np.testing.assert_array_equal(host(a), host(b))
    r.close()


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_staged_vector_stores_equal_scalar_stores(lor, dt):
    """Row-major dense saving with n_save a multiple of the staging group (4 saves in FP32,
    2 in FP64 for D = 3) goes through 16-byte vector stores; the SoA layout keeps scalar
    stores.  Same values, bit for bit, NaN slots and failures included."""
    P, U, T = workloads.lorenz_random(3000 + 7, seed=35, t1=2.0)
    T[::11, 1] = 0.0          # zero-length spans
    T[5::13, 0] = 0.5         # saves before t0 are NaN
    P[3, 0] = np.nan          # a failing trajectory
    sv = np.concatenate([[-0.5, 0.0], np.linspace(0.1, 2.0, 9), [2.5]])  # 12 save times
    kw = dict(abstol=1e-6, reltol=1e-6, saveat=sv, dense=True)
    o1, s1, _ = lor.solve(dev(P, dt), dev(U, dt), dev(T, dt), alg="tsit5", **kw)
    t = lambda a: dev(np.ascontiguousarray(a.T), dt)
    o2, s2, _ = lor.solve(t(P), t(U), t(T), alg="tsit5", layout="soa", **kw)
    a, b = host(o1), np.transpose(host(o2), (2, 0, 1))
    np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
    np.testing.assert_array_equal(np.nan_to_num(a), np.nan_to_num(b))
    np.testing.assert_array_equal(s1.cpu().numpy(), s2.cpu().numpy())
    assert s1.cpu().numpy()[3] != 0


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_dense_saves_equal_across_schedules(lor, dt):
    """The direct schedule and the persistent one (one and two trajectories per thread, a
    refilled warp) give the same dense saves bit for bit, in both layouts, with NaN slots,
    zero-length spans, a save at tf and a failing trajectory; n_save is not a multiple of the
    staging group, so the rows go out with scalar stores."""
    P, U, T = workloads.lorenz_random(5000 + 3, seed=36, t1=10.0)
    T[::11, 1] = 0.0          # zero-length spans
    T[5::13, 0] = 0.5         # saves before t0 are NaN
    P[3, 0] = np.nan          # a failing trajectory
    sv = np.concatenate([[-0.5, 0.0], np.linspace(0.05, 10.0, 200), [12.0]])
    kw = dict(abstol=1e-6, reltol=1e-6, saveat=sv, dense=True)
    d = lambda a: dev(a, dt)
    ref, rst, _ = lor.solve(d(P), d(U), d(T), alg="tsit5", schedule="direct", **kw)
    r = host(ref)
    assert int(rst.cpu().numpy()[3]) != 0 and np.isnan(r[3, 3:]).all()
    for tpt in (1, 2):
        out, st, _ = lor.solve(d(P), d(U), d(T), alg="tsit5", schedule="persistent", tpt=tpt, **kw)
        o = host(out)
        np.testing.assert_array_equal(np.isnan(o), np.isnan(r))
        np.testing.assert_array_equal(np.nan_to_num(o), np.nan_to_num(r))
        np.testing.assert_array_equal(st.cpu().numpy(), rst.cpu().numpy())
    t = lambda a: d(np.ascontiguousarray(a.T))
    o2, _, _ = lor.solve(t(P), t(U), t(T), alg="tsit5", layout="soa", schedule="persistent", **kw)
    o2 = np.transpose(host(o2), (2, 0, 1))
    np.testing.assert_array_equal(np.nan_to_num(o2), np.nan_to_num(r))


def test_dense_and_record_take_at_most_512_threads_per_block(lor):
    """The staged kernels keep their shared memory under the default 48 KB with at most 512
    threads per block: a larger block is refused before launch (no kernel runs), 512 works."""
    from paper_2304_06835_gb300 import EnsError
    P, U, T = workloads.lorenz_random(1000, seed=37, t1=1.0)
    kw = dict(abstol=1e-6, reltol=1e-6, saveat=SV, dense=True)
    for sched in ("direct", "persistent"):
        with pytest.raises(EnsError):
            lor.solve(dev(P), dev(U), dev(T), alg="tsit5", schedule=sched, block=1024, **kw)
        a, _, _ = lor.solve(dev(P), dev(U), dev(T), alg="tsit5", schedule=sched, block=512, **kw)
        b, _, _ = lor.solve(dev(P), dev(U), dev(T), alg="tsit5", schedule=sched, block=128, **kw)
        np.testing.assert_array_equal(host(a), host(b))
    cap = 16
    with pytest.raises(EnsError):
        lor.solve_steps(dev(P), dev(U), dev(T), cap, abstol=1e-6, reltol=1e-6, block=1024)
