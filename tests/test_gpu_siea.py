"""GPU parity of the weak order 2 stochastic Runge-Kutta step (GPUSIEA, Sec. 5.2.2) through
the C ABI, against the CPU oracle on the same Philox streams (Euler-Maruyama's convention:
step k uses normal k of the trajectory's stream, trajectory = index_offset + i):

* GBM in FP64 against the oracle to 1e-12 (state-vector relative, as Euler-Maruyama), with
  save times and a ragged N; FP32 against the oracle's FP64 arithmetic on the FP32 normal
  stream to 1e-5;
* the GPU ensemble's mean and second moment at 2^20 paths within 5 standard errors of the
  scheme's exact discrete moments E X_n = X0 m1^n, E X_n^2 = X0^2 m2^n with
  m1 = 1 + mu h + mu^2 h^2 / 2, m2 = m1^2 + sigma^2 h (1 + mu h)^2 + sigma^4 h^2 / 2;
* models without diagonal noise are refused; schedules change no result.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def dev(a, dt=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def normwise(out, ref):
    out = out.reshape(out.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.abs(out - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1.0)


@pytest.fixture(scope="module")
def gbm():
    from paper_2304_06835_gb300 import EnsembleSolver
    s = EnsembleSolver("gbm")
    yield s
    s.close()


@pytest.mark.parametrize("N", [1, 33, 4097])
def test_fp64_matches_oracle(gbm, N):
    P, U, T = workloads.gbm_random(N, seed=40 + N)
    sv = [0.0, 0.25, 0.5005, 1.0]
    ref, rs, rst = oracle.solve("gbm", "siea", P, U, T, dt=1e-3, seed=5, index_offset=11,
                                saveat=sv)
    out, st, stats = gbm.solve(dev(P), dev(U), dev(T), alg="siea", dt=1e-3, seed=5,
                               index_offset=11, saveat=sv, want_stats=True)
    o = out.cpu().numpy()
    assert normwise(o, ref).max() <= 1e-12
    assert np.all(st.cpu().numpy() == 0) and np.all(rs == 0)
    np.testing.assert_array_equal(stats.cpu().numpy().T, rst.astype(np.int32))


def test_fp32_matches_oracle_on_the_fp32_stream(gbm):
    P, U, T = workloads.gbm_random(4096, seed=44)
    P = P.astype(np.float32).astype(np.float64)
    ref, _, _ = oracle.solve("gbm", "siea", P, U, T, dt=1e-3, seed=6, precision="f64_f32stream")
    out, st, _ = gbm.solve(dev(P, torch.float32), dev(U, torch.float32), dev(T, torch.float32),
                           alg="siea", dt=1e-3, seed=6)
    assert normwise(out.cpu().double().numpy(), ref).max() <= 1e-5


def test_exact_discrete_moments(gbm):
    M, mu, sig, h, n = 1 << 20, 0.4, 0.5, 1e-2, 100
    P = np.tile([mu, sig], (M, 1))
    out, st, _ = gbm.solve(dev(P), dev(np.ones((M, 1))), dev(np.tile([0.0, n * h], (M, 1))),
                           alg="siea", dt=h, seed=2024)
    x = out.cpu().numpy()[:, 0]
    m1 = 1 + mu * h + mu * mu * h * h / 2
    m2 = m1 * m1 + sig * sig * h * (1 + mu * h) ** 2 + sig ** 4 * h * h / 2
    assert abs(x.mean() - m1 ** n) < 5 * x.std() / np.sqrt(M)
    assert abs((x * x).mean() - m2 ** n) < 5 * (x * x).std() / np.sqrt(M)


def test_refusals_and_schedules(gbm):
    from paper_2304_06835_gb300 import EnsError, EnsembleSolver
    c = EnsembleSolver("crn")
    P, U, T = workloads.crn_random(8, seed=1, t1=1.0)
    with pytest.raises(EnsError):
        c.solve(dev(P), dev(U), dev(T), alg="siea", dt=0.1, seed=1)
    c.close()
    P, U, T = workloads.gbm_random(3001, seed=45)
    res = []
    for kw in (dict(schedule="direct"), dict(schedule="persistent", order="index"),
               dict(schedule="persistent", order="cost", tpt=2)):
        o, _, _ = gbm.solve(dev(P, torch.float32), dev(U, torch.float32), dev(T, torch.float32),
                            alg="siea", dt=1e-3, seed=3, **kw)
        res.append(o.cpu().numpy())
    for r in res[1:]:
        np.testing.assert_array_equal(r, res[0])
