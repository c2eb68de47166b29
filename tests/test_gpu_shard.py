"""Work estimates and sharding on the GPU path (through the C ABI):

* ens_cost_keys: for fixed-step methods the key is the step count (tf - t0) / dt exactly;
  for adaptive Tsit5 on the headline parameter distribution with spans tf ~ U[1, 100] it
  ranks trajectories by their true attempt counts (Spearman correlation >= 0.8 against the
  solve's own counters; measured 0.84 -- the key sees the starting step, not the chaotic
  growth of |u| that later sets the step size);
* solve_sharded with the CUDA solver as the per-range solve (one rank, LPT over chunks of the
  cost keys, so every chunk runs with its own index_offset): the gathered result equals one
  solve of the whole ensemble bit for bit, SDE noise streams included.
"""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


def dev(a, dt=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def test_cost_keys_fixed_step_exact():
    from paper_2304_06835_gb300 import EnsembleSolver
    s = EnsembleSolver("gbm")
    P, U, T = workloads.gbm_random(5000, seed=4)
    T[:, 1] = np.random.default_rng(1).uniform(0.5, 2.0, len(T))
    keys = s.cost_keys(dev(P), dev(U), dev(T), alg="em", dt=1e-3, seed=1).cpu().numpy()
    np.testing.assert_array_equal(keys, ((T[:, 1] - T[:, 0]) / 1e-3).astype(np.float32))
    s.close()


def test_cost_keys_rank_adaptive_work():
    from scipy.stats import spearmanr

    from paper_2304_06835_gb300 import EnsembleSolver
    s = EnsembleSolver("lorenz")
    P, U, T = workloads.lorenz_random(8192, seed=2, t1=10.0)
    T[:, 1] = np.random.default_rng(3).uniform(1.0, 100.0, len(T))  # uneven spans
    args = (dev(P, torch.float32), dev(U, torch.float32), dev(T, torch.float32))
    keys = s.cost_keys(*args, alg="tsit5", abstol=1e-5, reltol=1e-5).cpu().numpy()
    _, _, stats = s.solve(*args, alg="tsit5", abstol=1e-5, reltol=1e-5, want_stats=True)
    attempts = stats.cpu().numpy()[:2].sum(axis=0)
    rho = spearmanr(keys, attempts).correlation
    print("Spearman(cost key, attempts) = %.3f" % rho)
    assert rho >= 0.8
    s.close()


@pytest.mark.parametrize("case", ["gbm_em", "lorenz_tsit5"])
def test_solve_sharded_gpu_equals_one_solve(case):
    from paper_2304_06835_gb300 import EnsembleSolver, solve_sharded
    if case == "gbm_em":
        s = EnsembleSolver("gbm")
        P, U, T = workloads.gbm_random(30001, seed=4)
        kw = dict(alg="em", dt=1e-3, seed=99)
    else:
        s = EnsembleSolver("lorenz")
        P, U, T = workloads.lorenz_random(30001, seed=2, t1=5.0)
        T[:, 1] = np.random.default_rng(4).uniform(0.5, 5.0, len(T))
        kw = dict(alg="tsit5", abstol=1e-6, reltol=1e-6)
    Pd, Ud, Td = dev(P), dev(U), dev(T)
    ref = s.solve(Pd, Ud, Td, want_stats=True, **kw)
    keys = s.cost_keys(Pd, Ud, Td, **kw)

    def fn(p, u, t, off):
        out, st, stats = s.solve(p, u, t, want_stats=True, index_offset=off, **kw)
        return out, st, stats.T.contiguous()

    out, st, stats = solve_sharded(fn, Pd, Ud, Td, costs=keys, chunk=4099)
    torch.cuda.synchronize()
    assert torch.equal(out, ref[0]) and torch.equal(st, ref[1])
    assert torch.equal(stats, ref[2].T)
    s.close()
