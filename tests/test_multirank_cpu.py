"""The multi-rank path on CPU ranks (gloo, world size 2): each rank solves its own shard
(weak scaling, no collective on the data path) and the job time is the maximum over the
ranks; the reference arm prints from rank 0 only; the moments of sharded ensembles merge
across the ranks (the one exchange step, an all-gather after the solve)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    t = bench.max_over_ranks(1.0 + rank * 0.5, world)
    # each rank's own end-to-end figure: 100 units/s on rank 0, 50 on rank 1, 10 units each
    e = bench.job_e2e({"value": 100.0 / (1 + rank), "unit": "u/s", "h2d_bytes_per_step": 8,
                       "d2h_bytes_per_step": 4}, 10, world)
    w = dict(bench.WORKLOADS["lorenz_adaptive_f32"], N=64)
    P, _, _ = bench.inputs_for(w, rank, world)
    wg = dict(bench.WORKLOADS["crn_em_f32"], N=64)
    q.put((rank, t, P, bench.shard_start(wg, rank, world), e))
    dist.destroy_process_group()


def test_max_over_ranks_and_shards_of_one_ensemble_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda r: r[0])
    assert res[0][1] == res[1][1] == 1.5           # every rank sees the slowest rank's time
    # the job's e2e: 20 units over the slower rank's 0.2 s per step, bytes of both ranks
    for r in res:
        assert r[4] == {"value": 100.0, "unit": "u/s", "h2d_bytes_per_step": 16,
                        "d2h_bytes_per_step": 8}
    sys.path.insert(0, ROOT)
    import bench
    whole, _, _ = bench.inputs_for(dict(bench.WORKLOADS["lorenz_adaptive_f32"], N=128))
    # the two contiguous halves of one ensemble of N x world trajectories
    np.testing.assert_array_equal(res[0][2], whole[:64])
    np.testing.assert_array_equal(res[1][2], whole[64:])
    assert (res[0][3], res[1][3]) == (0, 64)        # SDE streams by the global index


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(30500 + os.getpid() % 1000),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--workload", "lorenz_adaptive_f64"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"


def _local_moments(x):
    """A rank's (mean, M2, n) of its own shard, as ens_moments forms them on the GPU."""
    m = x.mean(0)
    return np.concatenate([m, ((x - m) ** 2).sum(0), [len(x)]])


def _moments_rank(rank, world, port, q, offset):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    from paper_2304_06835_gb300 import combine_moments
    x = offset + np.random.default_rng(11).lognormal(0.3, 0.8, size=(1001, 4))  # the ensemble
    mine = x[rank * 600:(rank + 1) * 600]                       # uneven contiguous shards
    n, mean, var = combine_moments(torch.tensor(_local_moments(mine), dtype=torch.float64))
    q.put((rank, float(n), np.asarray(mean), np.asarray(var)))
    dist.destroy_process_group()


@pytest.mark.parametrize("offset", [0.0, 1e8])
def test_moments_exchange_gloo(offset):
    """The exchange step of a sharded SDE ensemble: every rank gathers the others' (mean, M2,
    n) and merges them into the whole ensemble's count, mean and unbiased variance.  With an
    offset of 1e8 (|mean| / std ~ 1e8) raw power sums would lose the variance entirely; the
    merged form keeps it."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31500 + os.getpid() % 1000 + (7 if offset else 0)
    procs = [ctx.Process(target=_moments_rank, args=(r, 2, port, q, offset)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x = offset + np.random.default_rng(11).lognormal(0.3, 0.8, size=(1001, 4))
    for _, n, mean, var in res:
        assert n == 1001
        np.testing.assert_allclose(mean, x.mean(0), rtol=1e-13)
        np.testing.assert_allclose(var, x.var(0, ddof=1), rtol=1e-9)


def test_merge_moments_single_process_and_errors():
    """Without a process group the one rank's moments are used as they are; a merge of many
    uneven groups in order equals the whole; fewer than two trajectories raise."""
    from paper_2304_06835_gb300 import combine_moments, merge_moments
    x = np.random.default_rng(12).normal(2.0, 3.0, size=(777, 3))
    mom = torch.tensor(_local_moments(x))
    before = mom.clone()
    n, mean, var = combine_moments(mom)
    assert float(n) == 777
    np.testing.assert_allclose(mean, x.mean(0), rtol=1e-13)
    np.testing.assert_allclose(var, x.var(0, ddof=1), rtol=1e-12)
    assert torch.equal(mom, before)
    cuts = [0, 1, 2, 50, 51, 400, 777]
    parts = np.stack([_local_moments(x[a:b]) for a, b in zip(cuts[:-1], cuts[1:])])
    n2, mean2, var2 = merge_moments(parts)
    np.testing.assert_allclose(mean2, x.mean(0), rtol=1e-13)
    np.testing.assert_allclose(var2, x.var(0, ddof=1), rtol=1e-12)
    empty = np.zeros((2, 7))
    with pytest.raises(ValueError):
        merge_moments(empty)
    with pytest.raises(ValueError):
        merge_moments(_local_moments(x[:1]))
