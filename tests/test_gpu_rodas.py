"""GPU parity of Rodas4 and Rodas5P (Sec. 5.2.1: GPURodas4, GPURodas5P) through the C ABI,
against the CPU oracle (which steps the standard form of the methods, the kernels the
transformed form of the published coefficients):

* one accepted attempt of the adaptive kernel equals one oracle step from the same state
  (Robertson and Orego: 1e-11 relative, the stiff W; Lorenz and GBM: 1e-12 for Rodas4 and
  2e-11 for Rodas5P, whose transformed coefficients (|c_ij| up to ~170) make its stage sums
  cancel: the transformed form alone, emulated in FP64 on the host, differs from the
  oracle's standard form by up to 8.3e-12 on these GBM steps).  Random states with large
  stiff steps can make a step explode (stage values past 1e40); only steps that the oracle
  keeps bounded are compared (the kernel forms the error ratio in FP32 and reports the
  exploding ones as non-finite);
* Robertson over [0, 1e5] (the stiff benchmark configuration, FP64, tol 1e-6, h0 = 1e-4, 10
  log-spaced save times): every trajectory within 10x tol of a tol-1e-12 Rodas5P reference and
  of the oracle at the same tolerance, with the GPU's largest error against the reference no
  more than 5 % above the oracle's; the linear invariant y1 + y2 + y3 = 1 holds to 1e-10;
  f evaluations 1 + S per attempt.  Identical (accepted, rejected) counts: Rodas4 rejects no
  step here and matches on >= 95 % (measured 99.6 %); Rodas5P rejects ~0.1 step per
  trajectory, at the stiff steady state where its error estimate is round-off and the two
  forms' rounding flips decisions, and matches on >= 65 % (measured 71 %).  On identical
  counts the two agree to 0.15 of the tolerance (measured 0.0002 and 0.096);
* FP32 against the oracle's FP32 mode, with the oracle's FP64 mode as yardstick (as for
  Rosenbrock23);
* the paper's stiff test models (Orego, HIRES, POLLU) at tol 1e-6 under both methods: as
  close to a tol-1e-10 reference as the oracle at the same tolerance (within 3x its error
  plus 10x the tolerance), identical counts on >= 80 %, within 0.1 tol on those;
* the schedules (direct, persistent in index and cost order) give identical results.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

ALGS = ["rodas4", "rodas5p"]
STAGES = {"rodas4": 6, "rodas5p": 8}


def dev(a, dt=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().double().numpy()


@pytest.fixture(scope="module")
def S():
    from paper_2304_06835_gb300 import EnsembleSolver
    return {k: EnsembleSolver(k) for k in ("lorenz", "robertson", "gbm", "orego", "hires",
                                            "pollu")}


@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("rhs", ["robertson", "lorenz", "gbm", "orego"])
def test_single_step_parity(S, alg, rhs):
    rng = np.random.default_rng(8)
    D, _ = oracle.DIMS[oracle.RHS[rhs]]
    n = 256
    if rhs == "robertson":
        U = np.abs(rng.normal(0, 1, (n, 3))) * [1, 1e-5, 0.1]
        P = workloads.ROBERTSON_K0 * np.exp(rng.uniform(-0.1, 0.1, (n, 3)))
        hs = 10.0 ** rng.uniform(-4, 2, n)
    elif rhs == "lorenz":
        U = rng.normal(0, 5, (n, 3))
        P = np.stack([rng.uniform(8, 12, n), rng.uniform(0, 28, n), rng.uniform(2, 3, n)], 1)
        hs = 10.0 ** rng.uniform(-4, -1.5, n)
    elif rhs == "gbm":
        U = rng.uniform(0.5, 2, (n, 1))
        P = np.stack([rng.uniform(-2, 2, n), np.zeros(n)], 1)
        hs = 10.0 ** rng.uniform(-3, 1, n)
    else:
        P0, U0, _ = workloads.stiff("orego", n, seed=5, t1=1.0)
        P, U = P0, U0 * rng.uniform(0.5, 2.0, (n, 3))
        hs = 10.0 ** rng.uniform(-5, -2, n)
    ref = np.stack([oracle.step(rhs, alg, U[i], P[i], 0.0, hs[i])[0] for i in range(n)])
    keep = np.abs(ref).max(axis=1) <= 1e3 * np.maximum(np.abs(U).max(axis=1), 1.0)
    assert keep.mean() >= 0.5
    T = np.stack([np.zeros(n), hs], 1)
    g, st, stats = S[rhs].solve(dev(P), dev(U), dev(T), alg=alg, abstol=1e20, reltol=1e20,
                                dt0=1e3, want_stats=True)
    o = host(g)[keep]
    gs = stats.cpu().numpy()
    assert np.all(gs[0] == 1) and np.all(gs[1] == 0)
    assert np.all(gs[2] == 1 + STAGES[alg])
    assert np.all(st.cpu().numpy()[keep] == 0)
    ref = ref[keep]
    e = np.abs(o - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1e-300)
    bound = 1e-11 if rhs in ("robertson", "orego") else (2e-11 if alg == "rodas5p" else 1e-12)
    assert e.max() <= bound, e.max()


@pytest.mark.parametrize("alg", ALGS)
def test_robertson_fp64(S, alg):
    P, U, T = workloads.robertson_random(512, seed=31)
    tol = dict(abstol=1e-6, reltol=1e-6)
    sv = np.logspace(-4, 5, 10)
    ref, _, rst = oracle.solve("robertson", alg, P, U, T, dt0=1e-4, saveat=sv, **tol)
    fine, _, _ = oracle.solve("robertson", "rodas5p", P, U, T, abstol=1e-12, reltol=1e-12,
                              dt0=1e-8, saveat=sv)
    out, st, stats = S["robertson"].solve(dev(P), dev(U), dev(T), alg=alg, dt0=1e-4,
                                          saveat=sv, want_stats=True, **tol)
    o = host(out)
    assert int(st.abs().sum()) == 0
    unit = lambda x: (x / (1e-6 + 1e-6 * np.abs(fine))).reshape(len(P), -1).max(axis=1)
    e_orc, e_gpu = unit(np.abs(ref - fine)), unit(np.abs(o - fine))
    gs = stats.cpu().numpy().T
    same = np.all(gs[:, :2] == rst[:, :2], axis=1)
    d = unit(np.abs(o - ref))
    print("Robertson %s FP64: identical counts %.3f; GPU - oracle on those max %.3g tol; "
          "error vs reference GPU max %.3g, oracle max %.3g" % (alg, same.mean(), d[same].max(),
                                                               e_gpu.max(), e_orc.max()))
    assert same.mean() >= (0.95 if alg == "rodas4" else 0.65)
    assert d[same].max() <= 0.15
    assert e_gpu.max() <= 1.05 * e_orc.max()
    assert e_gpu.max() <= 10 and np.all(np.abs(o - ref) <= 10 * (1e-6 + 1e-6 * np.abs(ref)))
    assert np.all(gs[:, 2] == 1 + STAGES[alg] * (gs[:, 0] + gs[:, 1]))
    assert np.abs(o.sum(axis=2) - 1).max() < 1e-10


@pytest.mark.parametrize("alg", ALGS)
def test_robertson_fp32_against_fp32_oracle(S, alg):
    P, U, T = workloads.robertson_random(256, seed=33)
    P = P.astype(np.float32).astype(np.float64)
    sv = np.logspace(-4, 5, 10)
    tol = dict(abstol=1e-8, reltol=1e-4)
    o32, rs, _ = oracle.solve("robertson", alg, P, U, T, dt0=1e-4, saveat=sv, precision="f32",
                              **tol)
    o64, _, _ = oracle.solve("robertson", alg, P, U, T, dt0=1e-4, saveat=sv, **tol)
    out, st, _ = S["robertson"].solve(dev(P, torch.float32), dev(U, torch.float32),
                                      dev(T, torch.float32), alg=alg, dt0=1e-4, saveat=sv,
                                      **tol)
    o = host(out)
    assert int(st.abs().sum()) == 0 and np.all(rs == 0)
    unit = lambda x: (x / (1e-8 + 1e-4 * np.abs(o32))).reshape(len(P), -1).max(axis=1)
    d, d_ref = unit(np.abs(o - o32)), unit(np.abs(o64 - o32))
    print("Robertson %s FP32: GPU - FP32 oracle median %.3g max %.3g tol; FP64 oracle - FP32 "
          "oracle median %.3g max %.3g tol" % (alg, np.median(d), d.max(), np.median(d_ref),
                                               d_ref.max()))
    assert np.median(d) <= 3 * np.median(d_ref) + 1e-3
    assert d.max() <= 3 * d_ref.max() + 1e-3


@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("model,N", [("orego", 300), ("hires", 300), ("pollu", 128)])
def test_stiff_models(S, alg, model, N):
    P, U, T = workloads.stiff(model, N, seed=21)
    tol = 1e-6
    ref, _, _ = oracle.solve(model, "rodas5p", P, U, T, abstol=1e-10, reltol=1e-10)
    same, sst, sstats = oracle.solve(model, alg, P, U, T, abstol=tol, reltol=tol)
    out, st, stats = S[model].solve(dev(P), dev(U), dev(T), alg=alg, abstol=tol, reltol=tol,
                                    want_stats=True)
    o = host(out)
    assert int(st.abs().sum()) == 0 and np.all(sst == 0)
    e_gpu, e_orc = np.abs(o - ref), np.abs(same - ref)
    assert np.all(e_gpu <= 3 * e_orc + 10 * (tol + tol * np.abs(ref)))
    g = stats.cpu().numpy().T
    eq = np.all(g[:, :2] == sstats[:, :2], axis=1)
    d = np.abs(o[eq] - same[eq]) / (tol + tol * np.abs(same[eq]))
    print("%s %s: identical counts %.3f, GPU - oracle on those max %.3g tol, error vs "
          "reference GPU %.3g oracle %.3g" % (model, alg, eq.mean(), d.max(), e_gpu.max(),
                                              e_orc.max()))
    assert eq.mean() >= 0.8
    assert d.max() <= 0.1


@pytest.mark.parametrize("alg", ALGS)
def test_schedules_identical(S, alg):
    P, U, T = workloads.robertson_random(3001, seed=34)
    T[:, 1] = np.random.default_rng(2).uniform(1.0, 1e4, len(T))
    res = []
    for kw in (dict(schedule="direct"), dict(schedule="persistent", order="index"),
               dict(schedule="persistent", order="cost"), dict(schedule="persistent", block=64)):
        o, st, stats = S["robertson"].solve(dev(P), dev(U), dev(T), alg=alg, abstol=1e-7,
                                            reltol=1e-7, dt0=1e-5, want_stats=True, **kw)
        res.append((host(o), st.cpu().numpy(), stats.cpu().numpy()))
    for r in res[1:]:
        for x, y in zip(r, res[0]):
            np.testing.assert_array_equal(x, y)
