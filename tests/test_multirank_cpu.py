"""The multi-rank path on CPU ranks (gloo, world size 2): each rank solves its own shard
(weak scaling, no collective on the data path) and the job time is the maximum over the
ranks; the reference arm prints from rank 0 only; the moment sums of sharded ensembles add up
across the ranks (the one exchange step, an all-reduce after the solve)."""
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
    w = dict(bench.WORKLOADS["lorenz_adaptive_f32"], N=64)
    P, _, _ = bench.inputs_for(w, rank)
    q.put((rank, t, P.sum()))
    dist.destroy_process_group()


def test_max_over_ranks_and_disjoint_shards_gloo():
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
    res.sort()
    assert res[0][1] == res[1][1] == 1.5           # every rank sees the slowest rank's time
    assert res[0][2] != res[1][2]                  # each rank draws its own shard


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


def _moments_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    from paper_2304_06835_gb300 import combine_moments
    x = np.random.default_rng(11).lognormal(0.3, 0.8, size=(1001, 4))  # the whole ensemble
    mine = x[rank::world]                                                # this rank's shard
    sums = torch.tensor(np.concatenate([mine.sum(0), (mine * mine).sum(0), [len(mine)]]),
                        dtype=torch.float64)
    n, mean, var = combine_moments(sums)
    q.put((rank, float(n), mean.numpy(), var.numpy()))
    dist.destroy_process_group()


def test_moments_all_reduce_gloo():
    """The exchange step of a sharded SDE ensemble: every rank adds the others' sums and
    obtains the whole ensemble's count, mean and unbiased variance."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31500 + os.getpid() % 1000
    procs = [ctx.Process(target=_moments_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x = np.random.default_rng(11).lognormal(0.3, 0.8, size=(1001, 4))
    for _, n, mean, var in res:
        assert n == 1001
        np.testing.assert_allclose(mean, x.mean(0), rtol=1e-13)
        np.testing.assert_allclose(var, x.var(0, ddof=1), rtol=1e-11)


def test_combine_moments_single_process():
    """Without a process group the sums are used as they are: count, mean and the unbiased
    variance of the ensemble, and the input tensor is not modified."""
    from paper_2304_06835_gb300 import combine_moments
    x = np.random.default_rng(12).normal(2.0, 3.0, size=(777, 3))
    sums = torch.tensor(np.concatenate([x.sum(0), (x * x).sum(0), [len(x)]]))
    before = sums.clone()
    n, mean, var = combine_moments(sums)
    assert float(n) == 777
    np.testing.assert_allclose(mean.numpy(), x.mean(0), rtol=1e-13)
    np.testing.assert_allclose(var.numpy(), x.var(0, ddof=1), rtol=1e-10)
    assert torch.equal(sums, before)
