"""ens_solve_noalloc: the solve for callers that must not allocate device memory (a framework
that owns all device memory through its pool, a real-time loop that cannot afford cudaMalloc's
implicit synchronisation, a plugin whose host forbids allocations).  Its scratch lives in one
fixed device array of the library instead of handle-owned buffers.

The results must equal those of ens_solve on the same inputs, on two calls in a row (the
shared scratch keeps the previous call's contents, so each call must clear what it needs).
This file is collected last so that a run stopping at the first failure has run every other
test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _dev(a, dt):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _noalloc(rhs_id, P, U, T, opts, out, status, stats):
    from paper_2304_06835_gb300 import _lib
    N = P.shape[-1]
    s = torch.cuda.current_stream().cuda_stream
    _lib.check(_lib.lib().ens_solve_noalloc(
        rhs_id, N, ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(U.data_ptr()),
        ctypes.c_void_p(T.data_ptr()), ctypes.byref(opts), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stats.data_ptr()),
        ctypes.c_void_p(s)))


@pytest.mark.parametrize("case", ["lorenz_adaptive_f32", "lorenz_adaptive_f64",
                                  "robertson_ros23_f64", "gbm_em_f32"])
def test_noalloc_matches_ens_solve_twice(case):
    from paper_2304_06835_gb300 import EnsembleSolver, _lib, make_opts
    if case.startswith("lorenz"):
        rhs, alg = "lorenz", "tsit5"
        P, U, T = workloads.lorenz_random(20000, seed=7, t1=3.0)
        T[:, 1] = np.random.default_rng(1).uniform(0.5, 3.0, len(T))
        kw = dict(abstol=1e-6, reltol=1e-6)
    elif case.startswith("robertson"):
        rhs, alg = "robertson", "ros23"
        P, U, T = workloads.robertson_random(4000, seed=8)
        kw = dict(abstol=1e-6, reltol=1e-6, dt0=1e-4)
    else:
        rhs, alg = "gbm", "em"
        P, U, T = workloads.gbm_random(30000, seed=9)
        kw = dict(dt=1e-3, seed=11)
    dt = torch.float32 if case.endswith("f32") else torch.float64
    # structure-of-arrays inputs, as the bench feeds them
    Pd, Ud, Td = _dev(P.T, dt), _dev(U.T, dt), _dev(T.T, dt)
    N = P.shape[0]
    D = U.shape[1]
    solver = EnsembleSolver(rhs)
    ref, ref_st, ref_stats = solver.solve(Pd, Ud, Td, alg=alg, layout="soa", want_stats=True,
                                          **kw)
    opts, keep = make_opts(alg, _lib.F32 if dt == torch.float32 else _lib.F64, "soa", **kw)
    for call in range(2):
        out = torch.full((D, N), float("nan"), dtype=dt, device="cuda")
        st = torch.full((N,), -1, dtype=torch.int8, device="cuda")
        stats = torch.full((3, N), -1, dtype=torch.int32, device="cuda")
        _noalloc(_lib.RHS[rhs], Pd, Ud, Td, opts, out, st, stats)
        torch.cuda.synchronize()
        # same kernels, same per-trajectory arithmetic: the outputs agree exactly, which is
        # within every tolerance the parity tests use
        assert torch.equal(out, ref), call
        assert torch.equal(st, ref_st), call
        assert torch.equal(stats, ref_stats), call
    del keep


@pytest.mark.parametrize("case", ["crn_em_f32", "ball_events_f64", "lorenz_dense_f32",
                                  "pollu_ros23_f64"])
def test_noalloc_new_models_and_options(case):
    """The newer models (8-noise CRN, the bouncing ball's events, POLLU's loop LU) and the
    dense saving through the allocation-free path: equal to ens_solve, twice in a row."""
    from paper_2304_06835_gb300 import EnsembleSolver, _lib, make_opts
    S = 0
    if case.startswith("crn"):
        rhs, alg = "crn", "em"
        P, U, T = workloads.crn_random(5000, seed=12, t1=50.0)
        kw = dict(dt=0.1, seed=3)
    elif case.startswith("ball"):
        rhs, alg = "ball", "tsit5"
        P, U, T = workloads.ball(5000, seed=13)
        kw = dict(abstol=1e-8, reltol=1e-8, dtmax=1.0)
    elif case.startswith("lorenz"):
        rhs, alg = "lorenz", "tsit5"
        P, U, T = workloads.lorenz_random(8000, seed=14, t1=2.0)
        sv = np.linspace(0.0, 2.0, 17)
        S = len(sv)
        kw = dict(abstol=1e-6, reltol=1e-6, saveat=sv, dense=True)
    else:
        rhs, alg = "pollu", "ros23"
        P, U, T = workloads.stiff("pollu", 512, seed=15, t1=5.0)
        kw = dict(abstol=1e-6, reltol=1e-6)
    dt = torch.float32 if case.endswith("f32") else torch.float64
    Pd, Ud, Td = _dev(P.T, dt), _dev(U.T, dt), _dev(T.T, dt)
    N, D = P.shape[0], U.shape[1]
    solver = EnsembleSolver(rhs)
    ref, ref_st, ref_stats = solver.solve(Pd, Ud, Td, alg=alg, layout="soa", want_stats=True,
                                          **kw)
    opts, keep = make_opts(alg, _lib.F32 if dt == torch.float32 else _lib.F64, "soa", **kw)
    for call in range(2):
        out = torch.full((S, D, N) if S else (D, N), float("nan"), dtype=dt, device="cuda")
        st = torch.full((N,), -1, dtype=torch.int8, device="cuda")
        stats = torch.full((3, N), -1, dtype=torch.int32, device="cuda")
        _noalloc(_lib.RHS[rhs], Pd, Ud, Td, opts, out, st, stats)
        torch.cuda.synchronize()
        assert torch.equal(torch.nan_to_num(out), torch.nan_to_num(ref)), call
        assert torch.equal(st, ref_st), call
        assert torch.equal(stats, ref_stats), call
    del keep
    solver.close()


def test_noalloc_first_call_accuracy_against_oracle():
    """The allocation-free path on its own, checked against the CPU oracle (FP64 fixed-step
    Tsit5 on the Lorenz sweep: state-vector error <= 1e-12)."""
    from paper_2304_06835_gb300 import _lib, make_opts
    P, U, T = workloads.lorenz_sweep(1024)
    ref, _, _ = oracle.solve("lorenz", "tsit5_fixed", P, U, T, dt=1e-3)
    dt = torch.float64
    Pd, Ud, Td = _dev(P.T, dt), _dev(U.T, dt), _dev(T.T, dt)
    opts, keep = make_opts("tsit5_fixed", _lib.F64, "soa", dt=1e-3, schedule="persistent",
                           order="cost")
    out = torch.empty((3, 1024), dtype=dt, device="cuda")
    st = torch.empty(1024, dtype=torch.int8, device="cuda")
    stats = torch.empty((3, 1024), dtype=torch.int32, device="cuda")
    for _ in range(2):
        _noalloc(_lib.RHS["lorenz"], Pd, Ud, Td, opts, out, st, stats)
        torch.cuda.synchronize()
        o = out.cpu().numpy().T
        err = np.abs(o - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1)
        assert err.max() <= 1e-12
        assert int(st.abs().sum()) == 0
    del keep


def test_noalloc_rejects_sizes_beyond_its_maximum():
    from paper_2304_06835_gb300 import _lib, make_opts
    opts, keep = make_opts("tsit5", _lib.F32, "soa")
    small = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(small.data_ptr())
    rc = _lib.lib().ens_solve_noalloc(_lib.RHS["lorenz"], (1 << 20) + 1, p, p, p,
                                      ctypes.byref(opts), p, None, None, None)
    assert rc == _lib.ENS_EINVAL
    assert b"ENS_NOALLOC_MAX_N" in _lib.lib().ens_last_error()
    del keep


def test_noalloc_at_its_maximum_size_allocates_nothing():
    """N = ENS_NOALLOC_MAX_N, persistent schedule with the longest-first order (the largest
    use of the fixed scratch: queue, permutation and bucket keys of every trajectory): equal
    to ens_solve twice in a row, and the device's free memory is the same before and after
    the second call (the first call may load the library's module on the device)."""
    from paper_2304_06835_gb300 import EnsembleSolver, _lib, make_opts
    N = 1 << 20
    P, U, T = workloads.lorenz_random(N, seed=16, t1=1.0)
    dt = torch.float32
    Pd, Ud, Td = _dev(P.T, dt), _dev(U.T, dt), _dev(T.T, dt)
    kw = dict(abstol=1e-5, reltol=1e-5, schedule="persistent", order="cost")
    solver = EnsembleSolver("lorenz")
    ref, ref_st, ref_stats = solver.solve(Pd, Ud, Td, alg="tsit5", layout="soa",
                                          want_stats=True, **kw)
    opts, keep = make_opts("tsit5", _lib.F32, "soa", **kw)
    out = torch.empty((3, N), dtype=dt, device="cuda")
    st = torch.empty((N,), dtype=torch.int8, device="cuda")
    stats = torch.empty((3, N), dtype=torch.int32, device="cuda")
    for call in range(2):
        out.fill_(float("nan"))
        st.fill_(-1)
        stats.fill_(-1)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        _noalloc(_lib.RHS["lorenz"], Pd, Ud, Td, opts, out, st, stats)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        if call == 1:
            assert free1 == free0, (free0, free1)
        assert torch.equal(out, ref), call
        assert torch.equal(st, ref_st), call
        assert torch.equal(stats, ref_stats), call
    del keep
    solver.close()


def test_noalloc_errors_equal_ens_solve():
    """Invalid arguments are refused with ens_solve's own error codes: both run the same
    checks before touching the device."""
    from paper_2304_06835_gb300 import EnsembleSolver, _lib, make_opts
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    cases = [("orego", make_opts("em", _lib.F64, "soa", dt=0.1)),
             ("crn", make_opts("tsit5", _lib.F64, "soa")),
             ("lorenz", make_opts("tsit5", _lib.F64, "soa", blocks_per_sm=65)),
             ("lorenz", make_opts("tsit5", _lib.F64, "soa", tpt=3)),
             ("lorenz", make_opts("tsit5_fixed", _lib.F64, "soa", dt=-1.0))]
    for rhs, (opts, keep) in cases:
        s = EnsembleSolver(rhs)
        rc_solve = _lib.lib().ens_solve(s.handle, 4, p, p, p, ctypes.byref(opts), p, None, None,
                                        None)
        rc_noalloc = _lib.lib().ens_solve_noalloc(_lib.RHS[rhs], 4, p, p, p, ctypes.byref(opts),
                                                  p, None, None, None)
        assert rc_solve != _lib.ENS_OK and rc_noalloc == rc_solve, (rhs, rc_solve, rc_noalloc)
        s.close()
        del keep
