"""One ensemble across several ranks (one process per GPU): the paper's MPI path scatters a
single ensemble over the nodes, solves the parts independently and gathers the solutions
(Sec. 6.3).  Trajectories are independent, so no collective runs during the solve.

* shard_plan splits the index space [0, N) into contiguous ranges per rank: with no costs,
  one balanced range each; with per-trajectory costs (ens_cost_keys: expected steps, times
  a per-model weight for mixed work), chunks of `chunk` consecutive trajectories go to the
  ranks by longest-processing-time-first (LPT: heaviest chunk first, each to the rank with
  the least load so far, ties to the lowest rank).  Every rank computes the same plan.
* solve_sharded runs the caller's per-range solve with index_offset = the range's start,
  so SDE noise streams are those of the unsharded ensemble, and either leaves the results
  sharded or gathers them to rank 0 in the global order (point-to-point sends: gloo for CPU
  tensors, NCCL for CUDA tensors).
"""
from __future__ import annotations

import heapq

import numpy as np
import torch


def _world(group=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def shard_plan(N, world, costs=None, chunk=65536):
    """Ranges [(start, end), ...] per rank (a list of `world` lists, each sorted by start).
    costs: None, or per-trajectory work estimates [N] (NumPy or torch, any device)."""
    N, world = int(N), int(world)
    if world < 1:
        raise ValueError("world must be >= 1")
    if costs is None:
        cuts = [N * r // world for r in range(world + 1)]
        return [[(cuts[r], cuts[r + 1])] if cuts[r + 1] > cuts[r] else [] for r in range(world)]
    c = costs.detach().cpu().numpy() if torch.is_tensor(costs) else np.asarray(costs)
    c = np.nan_to_num(c.astype(np.float64).reshape(-1), nan=0.0, posinf=0.0)
    if c.size != N:
        raise ValueError("costs must have N entries")
    chunk = max(1, int(chunk))
    starts = np.arange(0, N, chunk)
    loads = np.add.reduceat(c, starts) if N else np.zeros(0)
    order = sorted(range(len(starts)), key=lambda k: (-loads[k], k))  # heaviest first, stable
    heap = [(0.0, r) for r in range(world)]
    plan = [[] for _ in range(world)]
    for k in order:
        load, r = heapq.heappop(heap)
        a = int(starts[k])
        plan[r].append((a, min(a + chunk, N)))
        heapq.heappush(heap, (load + float(loads[k]), r))
    return [sorted(p) for p in plan]


def _as_tensor(x, device=None):
    if torch.is_tensor(x):
        return x if device is None else x.to(device)
    return torch.from_numpy(np.ascontiguousarray(x))


def solve_sharded(solve_fn, params, u0, tspan, *, costs=None, chunk=65536, gather=True,
                  group=None):
    """Solve this rank's part of one ensemble.

    params [N, P], u0 [N, D], tspan [N, 2]: the whole ensemble, trajectory-major (NumPy or
    torch; every rank passes the same).  solve_fn(params, u0, tspan, index_offset) solves
    one contiguous range and returns a tuple of arrays whose first axis is the trajectory
    (e.g. out [n, D], status [n], stats [n, 3]).
    gather=True: rank 0 returns the tuple for all N trajectories in the global order (the
    other ranks return None).  gather=False: every rank returns its ranges as a list of
    (start, end, outputs)."""
    rank, world = _world(group)
    N = int(params.shape[0])
    plan = shard_plan(N, world, costs, chunk)
    mine = [(a, b, solve_fn(params[a:b], u0[a:b], tspan[a:b], a)) for a, b in plan[rank]]
    if not gather:
        return mine
    if world == 1:
        if len(mine) == 1:
            return tuple(_as_tensor(x) for x in mine[0][2])
        pieces = mine
    else:
        pieces = _gather_to_root(mine, plan, rank, world, group)
        if rank != 0:
            return None
    if not pieces:
        return None
    n_out = len(pieces[0][2])
    full = []
    for j in range(n_out):
        first = _as_tensor(pieces[0][2][j])
        buf = torch.empty((N,) + tuple(first.shape[1:]), dtype=first.dtype, device=first.device)
        for a, b, outs in pieces:
            buf[a:b] = _as_tensor(outs[j], buf.device)
        full.append(buf)
    return tuple(full)


def _gather_to_root(mine, plan, rank, world, group):
    """Rank 0 receives every rank's ranges (their outputs concatenated in range order, one
    message per output array); returns [(start, end, outputs)] for all ranges on rank 0."""
    import torch.distributed as dist
    # output shapes and dtypes: rank 0 describes them to everyone (it always holds a range
    # when N >= 1: the balanced plan gives it the first, LPT the heaviest chunk)
    desc = [None]
    if rank == 0:
        desc = [[(tuple(_as_tensor(x).shape[1:]), _as_tensor(x).dtype) for x in mine[0][2]]
                if mine else []]
    dist.broadcast_object_list(desc, src=0, group=group)
    desc = desc[0]
    if not desc:
        return []
    dev = _as_tensor(mine[0][2][0]).device if mine else None
    if rank != 0:
        for j, (shape, dtype) in enumerate(desc):
            if mine:
                cat = torch.cat([_as_tensor(o[2][j]) for o in mine]).contiguous()
                dist.send(cat, dst=dist.get_global_rank(group, 0) if group else 0, group=group)
        return []
    pieces = list(mine)
    for r in range(1, world):
        if not plan[r]:
            continue
        n_r = sum(b - a for a, b in plan[r])
        outs = []
        for shape, dtype in desc:
            buf = torch.empty((n_r,) + shape, dtype=dtype, device=dev)
            dist.recv(buf, src=dist.get_global_rank(group, r) if group else r, group=group)
            outs.append(buf)
        off = 0
        for a, b in plan[r]:
            pieces.append((a, b, tuple(o[off:off + (b - a)] for o in outs)))
            off += b - a
    return pieces
