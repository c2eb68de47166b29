"""One ensemble sharded across ranks (the paper's MPI scatter / gather of a single ensemble,
Sec. 6.3), on CPU ranks (gloo, world size 2) with the CPU oracle as the per-rank solve:

* shard_plan: every trajectory in exactly one contiguous range; with costs, LPT over chunks
  keeps every rank's load within one chunk of the average;
* solve_sharded gathered on rank 0 equals the unsharded solve bit for bit, for an adaptive
  ODE and for an SDE whose noise streams are indexed by the global trajectory number
  (index_offset = the range's start), with contiguous ranges and with LPT chunks;
* gather=False leaves each rank its own ranges, and they too equal the unsharded solve.
"""
import os
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plan_contiguous_and_lpt():
    from paper_2304_06835_gb300 import shard_plan
    for N, W in ((10, 3), (7, 8), (0, 2), (1_000_003, 4)):
        plan = shard_plan(N, W)
        assert len(plan) == W
        cover = sorted(r for p in plan for r in p)
        assert sum(b - a for a, b in cover) == N
        assert all(cover[k][1] == cover[k + 1][0] for k in range(len(cover) - 1))
        sizes = [sum(b - a for a, b in p) for p in plan]
        assert max(sizes) - min(sizes) <= 1
    rng = np.random.default_rng(3)
    c = rng.pareto(1.5, 100_001) + 1.0  # heavy-tailed work, as adaptive step counts are
    for W, chunk in ((2, 37), (3, 1000), (8, 4096)):
        plan = shard_plan(len(c), W, costs=c, chunk=chunk)
        cover = sorted(r for p in plan for r in p)
        assert cover[0][0] == 0 and cover[-1][1] == len(c)
        assert all(cover[k][1] == cover[k + 1][0] for k in range(len(cover) - 1))
        loads = [sum(c[a:b].sum() for a, b in p) for p in plan]
        biggest = max(c[a:b].sum() for a, b in cover)
        assert max(loads) <= np.mean(loads) + biggest
        assert plan == shard_plan(len(c), W, costs=c, chunk=chunk)  # deterministic


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import oracle
    import workloads
    from paper_2304_06835_gb300 import solve_sharded
    res = {}
    Pg, Ug, Tg = workloads.gbm_random(1001, seed=4)
    Pl, Ul, Tl = workloads.lorenz_random(501, seed=2, t1=3.0)
    Tl[:, 1] = np.random.default_rng(5).uniform(0.5, 3.0, len(Tl))  # uneven work

    def sde(P, U, T, off):
        return oracle.solve("gbm", "em", P, U, T, dt=1e-3, seed=77, index_offset=off,
                            nthreads=1)

    def ode(P, U, T, off):
        return oracle.solve("lorenz", "tsit5", P, U, T, abstol=1e-7, reltol=1e-7, nthreads=1)

    costs = Tl[:, 1] - Tl[:, 0]
    for name, fn, args, kw in (("sde", sde, (Pg, Ug, Tg), {}),
                               ("sde_lpt", sde, (Pg, Ug, Tg),
                                dict(costs=np.arange(1001.0) % 7, chunk=37)),
                               ("ode_lpt", ode, (Pl, Ul, Tl), dict(costs=costs, chunk=23))):
        g = solve_sharded(fn, *args, **kw)
        res[name] = None if g is None else [x.numpy() for x in g]
        res[name + "_sharded"] = [(a, b, [np.asarray(x) for x in o])
                                  for a, b, o in solve_sharded(fn, *args, gather=False, **kw)]
    q.put((rank, res))
    dist.destroy_process_group()


def test_solve_sharded_gloo_equals_unsharded():
    import oracle
    import workloads
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 32500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    Pg, Ug, Tg = workloads.gbm_random(1001, seed=4)
    Pl, Ul, Tl = workloads.lorenz_random(501, seed=2, t1=3.0)
    Tl[:, 1] = np.random.default_rng(5).uniform(0.5, 3.0, len(Tl))
    ref = {"sde": oracle.solve("gbm", "em", Pg, Ug, Tg, dt=1e-3, seed=77),
           "ode": oracle.solve("lorenz", "tsit5", Pl, Ul, Tl, abstol=1e-7, reltol=1e-7)}
    ref["sde_lpt"], ref["ode_lpt"] = ref["sde"], ref["ode"]
    for name in ("sde", "sde_lpt", "ode_lpt"):
        assert got[1][name] is None                       # only rank 0 holds the gather
        for x, r in zip(got[0][name], ref[name]):
            np.testing.assert_array_equal(x, r)
        covered = 0
        for rank in (0, 1):
            for a, b, outs in got[rank][name + "_sharded"]:
                covered += b - a
                for x, r in zip(outs, ref[name]):
                    np.testing.assert_array_equal(x, r[a:b])
        assert covered == len(ref[name][0])
    # the GBM solve needs its global stream index: without it the shards would differ
    P, U, T = workloads.gbm_random(1001, seed=4)
    wrong = oracle.solve("gbm", "em", P[500:], U[500:], T[500:], dt=1e-3, seed=77)[0]
    assert not np.array_equal(wrong, ref["sde"][0][500:])
