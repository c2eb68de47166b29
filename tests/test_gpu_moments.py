"""GPU check of the ensemble moments (ens_moments) through the C ABI:

* (mean, M2, n) equal NumPy's FP64 mean, sum of squared deviations and count of the same
  solve output in both layouts, FP32 and FP64, at every save slot, with and without a status
  mask, for a ragged N and for N = 0; two calls agree bit for bit (fixed merge order);
* values far from zero with a small spread (mean 1e6, standard deviation 1e-3: raw power
  sums would cancel every digit of the variance in FP64) keep the variance to 1e-9;
* Euler-Maruyama on GBM (Sec. 3.3, the linear SDE of the Appendix) at 2^20 trajectories: the
  mean and second moment of X_n lie within five standard errors of the exact moments of the
  discrete scheme, E X_n = X0 (1 + mu h)^n and E X_n^2 = X0^2 ((1 + mu h)^2 + sigma^2 h)^n.
"""
import math

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


def dev(a, dt=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def np_moments(o, st, slot, layout):
    """NumPy reference: o is the host copy of the solve output."""
    if layout == "rowmajor":
        x = o[:, slot, :] if o.ndim == 3 else o
    else:
        x = (o[slot] if o.ndim == 3 else o).T
    if st is not None:
        x = x[st == 0]
    m = x.mean(0)
    return np.concatenate([m, ((x - m) ** 2).sum(0), [len(x)]])


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
@pytest.mark.parametrize("layout", ["rowmajor", "soa"])
def test_moments_equal_numpy(dt, layout):
    from paper_2304_06835_gb300 import EnsembleSolver, ensemble_moments
    s = EnsembleSolver("lorenz")
    P, U, T = workloads.lorenz_random(3000 + 7, seed=81, t1=1.0)
    P[5, 0] = np.nan  # a failing trajectory: masked out by its status
    if layout == "soa":
        P, U, T = (np.ascontiguousarray(a.T) for a in (P, U, T))
    sv = np.linspace(0.0, 1.0, 5)
    out, st, _ = s.solve(dev(P, dt), dev(U, dt), dev(T, dt), alg="tsit5", layout=layout,
                         abstol=1e-6, reltol=1e-6, saveat=sv)
    torch.cuda.synchronize()
    o = out.cpu().double().numpy()
    sh = st.cpu().numpy()
    assert sh[5] != 0
    for slot in range(len(sv)):
        got = ensemble_moments(out, st, layout=layout, slot=slot).cpu().numpy()
        ref = np_moments(o, sh, slot, layout)
        # slot 0 is u0 = (1, 0, 0) for every trajectory: M2 = 0 exactly on both sides
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-9)
    a = ensemble_moments(out, layout=layout).cpu().numpy()        # no mask: NaN propagates
    assert np.isnan(a[:6]).all() and a[6] == len(sh)
    b = ensemble_moments(out, st, layout=layout).cpu().numpy()
    c = ensemble_moments(out, st, layout=layout).cpu().numpy()
    np.testing.assert_array_equal(b, c)
    s.close()


def test_empty_ensemble():
    from paper_2304_06835_gb300 import ensemble_moments
    z = ensemble_moments(torch.empty((0, 3), dtype=torch.float32, device="cuda"))
    np.testing.assert_array_equal(z.cpu().numpy(), np.zeros(7))


def test_large_mean_small_spread():
    from paper_2304_06835_gb300 import ensemble_moments, merge_moments
    rng = np.random.default_rng(5)
    x = 1e6 + 1e-3 * rng.normal(size=(500_001, 2))
    res = ensemble_moments(dev(x)).cpu().numpy()
    # exactly rounded references (NumPy's column mean of a row-major array adds in sequence
    # and is ~20 ulp off here)
    m = np.array([math.fsum(x[:, j]) / len(x) for j in range(2)])
    m2 = np.array([math.fsum((x[:, j] - m[j]) ** 2) for j in range(2)])
    np.testing.assert_allclose(res[:2], m, rtol=3e-16)
    np.testing.assert_allclose(res[2:4], m2, rtol=1e-9)
    n, mean, var = merge_moments(res)
    np.testing.assert_allclose(var, m2 / (len(x) - 1), rtol=1e-9)


def test_gbm_moments_match_the_discrete_scheme():
    from paper_2304_06835_gb300 import EnsembleSolver, combine_moments, ensemble_moments
    M = 1 << 20
    mu, sig, h, n = 0.4, 0.5, 1e-2, 100
    P = np.tile([mu, sig], (M, 1))
    g = EnsembleSolver("gbm")
    out, st, _ = g.solve(dev(P), dev(np.ones((M, 1))), dev(np.tile([0.0, 1.0], (M, 1))),
                         alg="em", dt=h, seed=2024)
    cnt, mean, var = combine_moments(ensemble_moments(out, st))  # one rank: no exchange
    x = out.cpu().numpy()[:, 0]
    m1 = (1 + mu * h) ** n
    m2 = ((1 + mu * h) ** 2 + sig * sig * h) ** n
    se1 = x.std() / np.sqrt(M)
    se2 = (x * x).std() / np.sqrt(M)
    assert float(cnt) == M
    assert abs(float(mean[0]) - m1) < 5 * se1
    e2 = float(var[0]) * (M - 1) / M + float(mean[0]) ** 2  # the second moment E X^2
    assert abs(e2 - m2) < 5 * se2
    np.testing.assert_allclose(float(var[0]), x.var(ddof=1), rtol=1e-9)
    g.close()
