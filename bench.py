"""Benchmark of the ensemble solver (one JSON line on stdout).

Default workload (the headline): Lorenz ensemble, N = 1,048,576 trajectories, rho~U[0,28],
sigma~U[8,12], beta~U[2,3], u0=(1,0,0), tspan [0,10], adaptive Tsit5 with PI control,
abstol = reltol = 1e-5, FP32, structure-of-arrays inputs resident in HBM.  One step = one
ensemble solve.  Metric: trajectories per second (whole job, all ranks).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Under torchrun (N > 1) every rank solves its own N-trajectory shard (weak scaling, no
collective on the data path); the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "Lorenz Tsit5 trajectories/s at N=1M, % FMA peak; surrogate vs solver at stated err"
SMS = 152
FP32_LANES = 128
SM_MAX_MHZ = 2070.0

# Algorithmic FP32 work per adaptive Tsit5 attempt on Lorenz (FMA-pipe instructions):
# stage combinations 81, six f evaluations 36, error estimate 21, scaled RMS norm 19,
# PI-controller arithmetic 3  -> 160 (selects, compares and clamps are not counted).
OPS_PER_ATTEMPT = {"tsit5": 160, "tsit5_fixed": 117, "rk4": 48, "ros23": 140, "em": 25}

WORKLOADS = {
    # name: (model, alg, dtype, N, t1, tol / dt)
    "lorenz_adaptive_f32": dict(rhs="lorenz", alg="tsit5", dtype="f32", N=1 << 20, t1=10.0,
                                tol=1e-5),
    "lorenz_adaptive_f64": dict(rhs="lorenz", alg="tsit5", dtype="f64", N=1 << 20, t1=10.0,
                                tol=1e-8),
    "lorenz_fixed_f32": dict(rhs="lorenz", alg="tsit5_fixed", dtype="f32", N=1 << 20, t1=1.0,
                             dt=1e-3),
    "robertson_ros23_f64": dict(rhs="robertson", alg="ros23", dtype="f64", N=1 << 18, t1=1e5,
                                tol=1e-6, dt0=1e-4),
}


def inputs_for(w, rank=0):
    N = w["N"]
    if w["rhs"] == "lorenz":
        if w["alg"] == "tsit5_fixed":
            P, U, T = workloads.lorenz_sweep(N, t1=w["t1"])
        else:
            P, U, T = workloads.lorenz_random(N, seed=2 + 1000 * rank, t1=w["t1"])
    elif w["rhs"] == "robertson":
        P, U, T = workloads.robertson_random(N, seed=3 + 1000 * rank, t1=w["t1"])
    else:
        P, U, T = workloads.gbm_random(N, seed=4 + 1000 * rank, t1=w["t1"])
    return P, U, T


def solve_kwargs(w):
    kw = {}
    if "tol" in w:
        kw.update(abstol=w["tol"], reltol=w["tol"])
    if "dt" in w:
        kw["dt"] = w["dt"]
    if "dt0" in w:
        kw["dt0"] = w["dt0"]
    return kw


# ------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.path = os.path.join("/tmp", "ens_clocks_%d.csv" % os.getpid())
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = np.array([float(r[1]) for r in rows if r[1].replace(".", "").isdigit()])
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = sm[sm > 0.5 * mx] if len(sm) else sm
        med = float(np.median(load)) if len(load) else float(np.median(sm))
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------------------------- oracle leg
def oracle_rate(w, budget_s=12.0):
    """Oracle (CPU, FP64, as it stands) on a bounded prefix of the same workload."""
    import oracle
    P, U, T = inputs_for(w)
    kw = solve_kwargs(w)
    nt = oracle.default_threads()
    n = min(w["N"], 4 * nt)
    t0 = time.perf_counter()
    oracle.solve(w["rhs"], w["alg"], P[:n], U[:n], T[:n], nthreads=nt, **kw)
    dt = time.perf_counter() - t0
    n2 = int(min(w["N"], max(n, n * budget_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oracle.solve(w["rhs"], w["alg"], P[:n2], U[:n2], T[:n2], nthreads=nt, **kw)
    dt = time.perf_counter() - t0
    return n2 / dt, n2, nt, dt


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    import oracle
    P, U, T = inputs_for(w)
    kw = solve_kwargs(w)
    nt = oracle.default_threads()
    rate, n, _, _ = oracle_rate(w, budget_s=4.0)
    n = max(1, int(rate * 3.0))  # each step ~3 s of CPU work
    for _ in range(args.warmup):
        oracle.solve(w["rhs"], w["alg"], P[:n], U[:n], T[:n], nthreads=nt, **kw)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve(w["rhs"], w["alg"], P[:n], U[:n], T[:n], nthreads=nt, **kw)
    el = time.perf_counter() - t0
    v = n * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "trajectories/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "N_sample": n, "N_full": w["N"]},
        "cpu_baseline": {"value": v, "unit": "trajectories/s", "cores": nt, "kind": "oracle",
                         "sample": "first %d trajectories of the %s workload per step"
                                   % (n, args.workload)},
        "e2e": {"value": v, "unit": "trajectories/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def e2e_rate(args, w, P, U, T, solver, stream, kw):
    """Trajectories/s through ens_solve_host: pinned host inputs copied to the device, the
    solve, and the outputs (final state + status) copied back, all inside the timed region."""
    import ctypes

    import torch

    import paper_2304_06835_gb300 as ens
    from paper_2304_06835_gb300 import _lib
    N = w["N"]
    npdt = np.float32 if w["dtype"] == "f32" else np.float64
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=npdt)).pin_memory()
    Pp, Up, Tp = pin(P.T), pin(U.T), pin(T.T)
    D = U.shape[1]
    outp = torch.empty((D, N), dtype=Pp.dtype).pin_memory()
    stp = torch.empty(N, dtype=torch.int8).pin_memory()
    o, keep = ens.make_opts(w["alg"], _lib.F32 if w["dtype"] == "f32" else _lib.F64, "soa",
                            schedule=args.schedule, block=args.block, tpt=args.tpt,
                            refill_min=args.refill, order=args.order, **kw)
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def host_step():
        _lib.check(_lib.lib().ens_solve_host(solver.handle, N, Pp.data_ptr(), Up.data_ptr(),
                                             Tp.data_ptr(), ctypes.byref(o), outp.data_ptr(),
                                             stp.data_ptr(), None, sptr))
    host_step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(steps):
        host_step()
    el = (time.perf_counter() - t0) / steps
    es = np.dtype(npdt).itemsize
    return {"value": N / el, "unit": "trajectories/s",
            "h2d_bytes_per_step": int(N * es * (P.shape[1] + D + 2)),
            "d2h_bytes_per_step": int(N * es * D + N)}


# ------------------------------------------------------------------------------- GPU leg
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="lorenz_adaptive_f32", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--tpt", type=int, default=0)
    ap.add_argument("--refill", type=int, default=0, help="persistent refill batch (0 = default)")
    ap.add_argument("--order", default="auto", choices=["auto", "index", "cost"])
    ap.add_argument("--schedule", default="auto")
    ap.add_argument("--n", type=int, default=0, help="override N (small profiling cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--probe", action="store_true", help="also measure FP32/FP64 FMA rates")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.n:
        w["N"] = args.n

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import paper_2304_06835_gb300 as ens
    from paper_2304_06835_gb300 import _lib

    dt_t = torch.float32 if w["dtype"] == "f32" else torch.float64
    P, U, T = inputs_for(w, rank)
    N = w["N"]
    dev = torch.device("cuda", local)
    Pd = torch.tensor(P.T.copy(), dtype=dt_t, device=dev)
    Ud = torch.tensor(U.T.copy(), dtype=dt_t, device=dev)
    Td = torch.tensor(T.T.copy(), dtype=dt_t, device=dev)
    D = U.shape[1]
    out = torch.empty((D, N), dtype=dt_t, device=dev)
    status = torch.empty(N, dtype=torch.int8, device=dev)
    stats = torch.empty((3, N), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    solver = ens.EnsembleSolver(w["rhs"])
    kw = solve_kwargs(w)
    stream = torch.cuda.current_stream(dev)

    def step():
        solver.solve(Pd, Ud, Td, alg=w["alg"], layout="soa", out=out, status=status, stats=stats,
                     schedule=args.schedule, block=args.block, tpt=args.tpt,
                     refill_min=args.refill, order=args.order, want_stats=True, **kw)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)  # L2 flush between timed solves (outside the events)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    tot_s = sum(ms) / 1e3
    if world > 1:
        t = torch.tensor([tot_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_s = float(t.item())
    value = N * world * args.steps / tot_s

    st = stats.cpu().numpy().astype(np.int64)
    attempts = int(st[0].sum() + st[1].sum())
    ok = int((status.cpu().numpy() == 0).sum())
    ops = attempts * OPS_PER_ATTEMPT[w["alg"]]
    launch_s = tot_s / args.steps
    achieved = ops / launch_s / 1e12
    peak_max = SMS * FP32_LANES * SM_MAX_MHZ * 1e6 / 1e12
    sm_mhz = clocks.get("sm_mhz") or SM_MAX_MHZ
    peak_clk = SMS * FP32_LANES * sm_mhz * 1e6 / 1e12
    bound = "alu"

    # e2e: the same solve through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        e2e = e2e_rate(args, w, P, U, T, solver, stream, kw)
    line = {
        "metric": METRIC, "value": value, "unit": "trajectories/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": 1e3 * launch_s,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": w["dtype"],
        "data": "synthetic",
        "config": {"workload": args.workload, "model": w["rhs"], "alg": w["alg"], "N": N,
                   "tspan": [0.0, w["t1"]], **{k: w[k] for k in ("tol", "dt", "dt0") if k in w},
                   "layout": "soa", "l2": "flushed between steps (256 MB write outside events)",
                   "parallelism": "dp%d" % world, "block": args.block, "tpt": args.tpt,
                   "schedule": args.schedule, "refill_min": args.refill,
                   "order": args.order},
        "wall_s": wall,
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak_max,
                     "unit": "T FP32-FMA-pipe instr/s", "frac": achieved / peak_max,
                     "frac_at_sampled_clock": achieved / peak_clk, "traffic": None,
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2070 MHz (derived)",
                     "ops_per_attempt": OPS_PER_ATTEMPT[w["alg"]],
                     "attempts_per_launch": attempts},
        "clocks": clocks,
        "gpu_launches": args.steps,
        "trajectories_ok": ok,
        "e2e": e2e,
    }
    if args.probe:
        import ctypes as C
        for dt_name, code in (("fp32", _lib.F32), ("fp64", _lib.F64)):
            r = C.c_double()
            iters = 20000 if code == _lib.F32 else 400
            _lib.check(_lib.lib().ens_probe_fma(code, iters, SMS * 8, 256, C.byref(r), None))
            line.setdefault("probe", {})[dt_name + "_fma_per_s"] = r.value
    if rank == 0 and not args.no_cpu_baseline:
        rate, n, nt, el = oracle_rate(w)
        line["cpu_baseline"] = {"value": rate, "unit": "trajectories/s", "cores": nt,
                                "kind": "oracle",
                                "sample": "first %d of the %d trajectories (%.1f s)" % (n, N, el)}
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
