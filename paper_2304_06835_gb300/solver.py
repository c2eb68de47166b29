"""Python front-end of the ensemble solver: torch tensors in, the C ABI does the work.

    solver = EnsembleSolver("lorenz")
    out, status, stats = solver.solve(params, u0, tspan, alg="tsit5", abstol=1e-8, reltol=1e-8)

Tensors must live on the CUDA device; torch supplies only memory and the stream.  Layouts:
  "rowmajor": params [N,P], u0 [N,D], tspan [N,2], out [N,D] (or [N,S,D] with saveat)
  "soa":      params [P,N], u0 [D,N], tspan [2,N], out [D,N] (or [S,D,N] with saveat)
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

_TORCH_DT = {torch.float32: _lib.F32, torch.float64: _lib.F64}
_NP_DT = {np.dtype(np.float32): _lib.F32, np.dtype(np.float64): _lib.F64}


def make_opts(alg="tsit5", dtype=_lib.F32, layout="rowmajor", dt=0.0, abstol=1e-6, reltol=1e-6,
              dt0=0.0, maxiters=1_000_000, saveat=None, seed=0, index_offset=0,
              schedule="auto", block=0, tpt=0, refill_min=0, order="auto", blocks_per_sm=0,
              dense=False, dtmax=0.0, step_cap=0, step_t=None, step_n=None,
              kernel_events=None):
    o = _lib.EnsOpts()
    _lib.lib().ens_opts_default(ctypes.byref(o))
    o.alg = _lib.ALG[alg] if isinstance(alg, str) else int(alg)
    o.dtype = dtype
    o.layout = _lib.LAYOUT[layout] if isinstance(layout, str) else int(layout)
    o.dt = float(dt)
    o.abstol = float(abstol)
    o.reltol = float(reltol)
    o.dt0 = float(dt0)
    o.maxiters = int(maxiters)
    keep = None
    if saveat is not None and len(saveat):
        keep = np.ascontiguousarray(saveat, dtype=np.float64)
        o.saveat = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        o.n_save = int(keep.size)
    o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    o.index_offset = int(index_offset)
    o.schedule = _lib.SCHED[schedule] if isinstance(schedule, str) else int(schedule)
    o.block = int(block)
    o.tpt = int(tpt)
    o.refill_min = int(refill_min)
    o.order = _lib.ORDER[order] if isinstance(order, str) else int(order)
    o.blocks_per_sm = int(blocks_per_sm)
    o.dense = 1 if dense else 0
    o.dtmax = float(dtmax)
    o.step_cap = int(step_cap)
    o.step_t = None if step_t is None else step_t.data_ptr()
    o.step_n = None if step_n is None else step_n.data_ptr()
    if kernel_events is not None:  # (start, stop) torch.cuda.Event, recorded around the kernel
        for e in kernel_events:
            if not e.cuda_event:  # torch creates the CUDA event at its first record
                e.record()
        o.kernel_start = kernel_events[0].cuda_event
        o.kernel_stop = kernel_events[1].cuda_event
    return o, keep


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class EnsembleSolver:
    """One solver handle for one right-hand side ("lorenz", "robertson", "gbm", "crn" or
    "ball"; the CRN takes alg="em" only, the bouncing ball alg="tsit5" only)."""

    def __init__(self, rhs: str):
        self.rhs = rhs
        self.rhs_id = _lib.RHS[rhs]
        self.D, self.P = _lib.DIMS[self.rhs_id]
        h = ctypes.c_void_p()
        _lib.check(_lib.lib().ens_create(ctypes.byref(h), self.rhs_id, self.D, self.P))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().ens_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def _shapes(self, N, S, layout, saved):
        D, P = self.D, self.P
        if layout == "rowmajor":
            return (N, P), (N, D), (N, 2), ((N, S, D) if saved else (N, D))
        return (P, N), (D, N), (2, N), ((S, D, N) if saved else (D, N))

    def solve(self, params, u0, tspan, alg="tsit5", *, layout="rowmajor", dt=0.0, abstol=1e-6,
              reltol=1e-6, dt0=0.0, maxiters=1_000_000, saveat=None, seed=0, index_offset=0,
              schedule="auto", block=0, tpt=0, refill_min=0, order="auto", blocks_per_sm=0,
              dense=False, dtmax=0.0, want_status=True, want_stats=False, out=None, status=None,
              stats=None, stream=None, kernel_events=None):
        """Solve the ensemble on the GPU (device tensors in and out).  dense=True (adaptive
        Tsit5 with saveat): save times take the step's dense output instead of cutting the
        steps, so the steps and final state are those of the solve without save times.
        dtmax > 0 caps adaptive steps."""
        if not (params.is_cuda and u0.is_cuda and tspan.is_cuda):
            raise ValueError("params, u0 and tspan must be CUDA tensors")
        if params.dtype not in _TORCH_DT or u0.dtype != params.dtype or tspan.dtype != params.dtype:
            raise ValueError("params, u0, tspan must share dtype float32 or float64")
        N = params.shape[0] if layout == "rowmajor" else params.shape[-1]
        S = len(saveat) if saveat is not None and len(saveat) else 1
        saved = saveat is not None and len(saveat) > 0
        sp, su, st, so = self._shapes(N, S, layout, saved)
        for name, t, shp in (("params", params, sp), ("u0", u0, su), ("tspan", tspan, st)):
            if tuple(t.shape) != shp or not t.is_contiguous():
                raise ValueError("%s must be contiguous with shape %s, got %s"
                                 % (name, shp, tuple(t.shape)))
        dev = params.device
        if out is None:
            out = torch.empty(so, dtype=params.dtype, device=dev)
        if want_status and status is None:
            status = torch.empty(N, dtype=torch.int8, device=dev)
        if want_stats and stats is None:
            stats = torch.empty((3, N), dtype=torch.int32, device=dev)
        o, keep = make_opts(alg, _TORCH_DT[params.dtype], layout, dt, abstol, reltol, dt0, maxiters,
                            saveat, seed, index_offset, schedule, block, tpt, refill_min, order,
                            blocks_per_sm, dense, dtmax, kernel_events=kernel_events)
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
        _lib.check(_lib.lib().ens_solve(self._h, N, _ptr(params), _ptr(u0), _ptr(tspan),
                                        ctypes.byref(o), _ptr(out), _ptr(status), _ptr(stats),
                                        ctypes.c_void_p(s)))
        del keep
        return out, status, stats

    def solve_steps(self, params, u0, tspan, cap, alg="tsit5", *, layout="rowmajor",
                    abstol=1e-6, reltol=1e-6, dt0=0.0, maxiters=1_000_000, dtmax=0.0,
                    schedule="auto", block=0, tpt=0, want_stats=False, stream=None):
        """Store every accepted step of an adaptive solve (the full solution): returns
        (t, u, n, status, stats) with u [N, cap, D] (SoA: [cap, D, N]) holding the state after
        k accepted steps (k = 0: u0), t [N, cap] (SoA [cap, N]) their times, n [N] = accepted
        steps + 1 (may exceed cap: the first cap entries are kept).  Entries past n are not
        written (left as allocated: NaN here)."""
        if not (params.is_cuda and u0.is_cuda and tspan.is_cuda):
            raise ValueError("params, u0 and tspan must be CUDA tensors")
        N = params.shape[0] if layout == "rowmajor" else params.shape[-1]
        dev = params.device
        D = self.D
        shp_u = (N, cap, D) if layout == "rowmajor" else (cap, D, N)
        shp_t = (N, cap) if layout == "rowmajor" else (cap, N)
        u = torch.full(shp_u, float("nan"), dtype=params.dtype, device=dev)
        t = torch.full(shp_t, float("nan"), dtype=params.dtype, device=dev)
        n = torch.empty(N, dtype=torch.int32, device=dev)
        status = torch.empty(N, dtype=torch.int8, device=dev)
        stats = torch.empty((3, N), dtype=torch.int32, device=dev) if want_stats else None
        o, keep = make_opts(alg, _TORCH_DT[params.dtype], layout, 0.0, abstol, reltol, dt0,
                            maxiters, None, 0, 0, schedule, block, tpt, 0, "auto", 0, False,
                            dtmax, cap, t, n)
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
        _lib.check(_lib.lib().ens_solve(self._h, N, _ptr(params), _ptr(u0), _ptr(tspan),
                                        ctypes.byref(o), _ptr(u), _ptr(status), _ptr(stats),
                                        ctypes.c_void_p(s)))
        del keep
        return t, u, n, status, stats

    def autotune(self, params, u0, tspan, alg="tsit5", *, layout="rowmajor", out=None,
                 status=None, stats=None, stream=None, **kw):
        """Time the candidate launch shapes on these inputs (the solve really runs) and cache
        the fastest for later solves with block = tpt = blocks_per_sm = 0.  Returns
        (block, tpt, blocks_per_sm, ms)."""
        N = params.shape[0] if layout == "rowmajor" else params.shape[-1]
        saveat = kw.get("saveat")
        saved = saveat is not None and len(saveat) > 0
        S = len(saveat) if saved else 1
        so = self._shapes(N, S, layout, saved)[3]
        dev = params.device
        if out is None:
            out = torch.empty(so, dtype=params.dtype, device=dev)
        o, keep = make_opts(alg, _TORCH_DT[params.dtype], layout, **kw)
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
        b, t, f, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        _lib.check(_lib.lib().ens_autotune(self._h, N, _ptr(params), _ptr(u0), _ptr(tspan),
                                           ctypes.byref(o), _ptr(out), _ptr(status), _ptr(stats),
                                           ctypes.c_void_p(s), ctypes.byref(b), ctypes.byref(t),
                                           ctypes.byref(f), ctypes.byref(ms)))
        del keep
        return b.value, t.value, f.value, ms.value

    def cost_keys(self, params, u0, tspan, alg="tsit5", *, layout="rowmajor", stream=None,
                  **kw):
        """Expected steps per trajectory (ens_cost_keys): a float32 tensor [N] on the inputs'
        device, the work estimate that balances shards across ranks (solve_sharded)."""
        N = params.shape[0] if layout == "rowmajor" else params.shape[-1]
        keys = torch.empty(N, dtype=torch.float32, device=params.device)
        o, keep = make_opts(alg, _TORCH_DT[params.dtype], layout, **kw)
        s = (torch.cuda.current_stream(params.device).cuda_stream if stream is None
             else stream.cuda_stream)
        _lib.check(_lib.lib().ens_cost_keys(self._h, N, _ptr(params), _ptr(u0), _ptr(tspan),
                                            ctypes.byref(o), _ptr(keys), ctypes.c_void_p(s)))
        del keep
        return keys

    # --------------------------------------------------------------- discrete adjoint
    def _adj_common(self, params, u0, tspan, layout):
        if not (params.is_cuda and u0.is_cuda and tspan.is_cuda):
            raise ValueError("params, u0 and tspan must be CUDA tensors")
        if params.dtype not in _TORCH_DT or u0.dtype != params.dtype or tspan.dtype != params.dtype:
            raise ValueError("params, u0, tspan must share dtype float32 or float64")
        N = params.shape[0] if layout == "rowmajor" else params.shape[-1]
        sp, su, st, so = self._shapes(N, 1, layout, False)
        for name, t, shp in (("params", params, sp), ("u0", u0, su), ("tspan", tspan, st)):
            if tuple(t.shape) != shp or not t.is_contiguous():
                raise ValueError("%s must be contiguous with shape %s, got %s"
                                 % (name, shp, tuple(t.shape)))
        return N, so

    @staticmethod
    def max_steps_of(tspan, dt, layout="rowmajor"):
        """Largest fixed-step count over the ensemble (reads tspan back to the host)."""
        span = (tspan[:, 1] - tspan[:, 0]) if layout == "rowmajor" else (tspan[1] - tspan[0])
        if span.numel() == 0:
            return 1
        return max(1, int(np.ceil(float(span.double().max().item()) / dt - 1e-12)))

    def ckpt_elems(self, N, max_steps, checkpoint_every=64):
        return int(_lib.lib().ens_adjoint_ckpt_elems(N, self.D, int(max_steps),
                                                     int(checkpoint_every)))

    def adjoint_forward(self, params, u0, tspan, alg="tsit5_fixed", *, dt, layout="rowmajor",
                        max_steps=None, checkpoint_every=64, out=None, ckpt=None, status=None,
                        stream=None):
        """Fixed-step solve that also stores checkpoints for `adjoint`.  Returns (out, ckpt,
        status, max_steps)."""
        N, so = self._adj_common(params, u0, tspan, layout)
        if max_steps is None:
            max_steps = self.max_steps_of(tspan, dt, layout)
        dev = params.device
        if out is None:
            out = torch.empty(so, dtype=params.dtype, device=dev)
        if ckpt is None:
            ckpt = torch.empty(max(1, self.ckpt_elems(N, max_steps, checkpoint_every)),
                               dtype=params.dtype, device=dev)
        if status is None:
            status = torch.empty(N, dtype=torch.int8, device=dev)
        o, keep = make_opts(alg, _TORCH_DT[params.dtype], layout, dt=dt)
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
        _lib.check(_lib.lib().ens_adjoint_forward(
            self._h, N, _ptr(params), _ptr(u0), _ptr(tspan), ctypes.byref(o), int(max_steps),
            int(checkpoint_every), _ptr(out), _ptr(ckpt), _ptr(status), ctypes.c_void_p(s)))
        del keep
        return out, ckpt, status, max_steps

    def adjoint(self, params, u0, tspan, grad_out, alg="tsit5_fixed", *, dt, layout="rowmajor",
                max_steps=None, checkpoint_every=64, ckpt=None, grad_p=None, grad_u0=None,
                stream=None):
        """dL/dp and dL/du0 of the fixed-step map given grad_out = dL/du(tf).  With ckpt=None
        the forward pass is rerun inside the library."""
        N, so = self._adj_common(params, u0, tspan, layout)
        if tuple(grad_out.shape) != so or grad_out.dtype != params.dtype or not grad_out.is_cuda:
            raise ValueError("grad_out must be a CUDA tensor of shape %s and dtype %s"
                             % (so, params.dtype))
        grad_out = grad_out.contiguous()
        if max_steps is None:
            max_steps = self.max_steps_of(tspan, dt, layout)
        dev = params.device
        if grad_p is None:
            grad_p = torch.empty_like(params)
        if grad_u0 is None:
            grad_u0 = torch.empty_like(u0)
        o, keep = make_opts(alg, _TORCH_DT[params.dtype], layout, dt=dt)
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
        _lib.check(_lib.lib().ens_adjoint(
            self._h, N, _ptr(params), _ptr(u0), _ptr(tspan), ctypes.byref(o), int(max_steps),
            int(checkpoint_every), _ptr(ckpt), _ptr(grad_out), _ptr(grad_p), _ptr(grad_u0),
            ctypes.c_void_p(s)))
        del keep
        return grad_p, grad_u0

    def solve_host(self, params, u0, tspan, alg="tsit5", *, layout="rowmajor", want_stats=False,
                   stream=None, **kw):
        """NumPy (host) arrays in and out; the library copies to and from the device."""
        params = np.ascontiguousarray(params)
        u0 = np.ascontiguousarray(u0, dtype=params.dtype)
        tspan = np.ascontiguousarray(tspan, dtype=params.dtype)
        if params.dtype not in _NP_DT:
            raise ValueError("dtype must be float32 or float64")
        N = params.shape[0] if layout == "rowmajor" else params.shape[-1]
        saveat = kw.get("saveat")
        saved = saveat is not None and len(saveat) > 0
        S = len(saveat) if saved else 1
        so = self._shapes(N, S, layout, saved)[3]
        out = np.empty(so, dtype=params.dtype)
        status = np.empty(N, dtype=np.int8)
        stats = np.empty((3, N), dtype=np.int32) if want_stats else None
        o, keep = make_opts(kw.pop("alg", alg), _NP_DT[params.dtype], layout, **kw)
        s = 0 if stream is None else stream.cuda_stream
        _lib.check(_lib.lib().ens_solve_host(
            self._h, N, params.ctypes.data, u0.ctypes.data, tspan.ctypes.data, ctypes.byref(o),
            out.ctypes.data, status.ctypes.data, None if stats is None else stats.ctypes.data,
            ctypes.c_void_p(s)))
        del keep
        return out, status, stats


def philox_words(seed, n_traj, n_calls, index_offset=0, device="cuda"):
    """uint32 words [n_calls, 4, n_traj] of the SDE streams (bit-exact Philox4x32-10)."""
    out = torch.empty((n_calls, 4, n_traj), dtype=torch.int32, device=device)
    s = torch.cuda.current_stream(out.device).cuda_stream
    _lib.check(_lib.lib().ens_philox4x32_10(int(seed), int(index_offset), int(n_traj),
                                            int(n_calls), _ptr(out), ctypes.c_void_p(s)))
    return out


def normals(seed, n_traj, n_per, dtype=torch.float32, index_offset=0, device="cuda"):
    """Standard normals [n_per, n_traj] that drive Euler-Maruyama (step k of trajectory j)."""
    out = torch.empty((n_per, n_traj), dtype=dtype, device=device)
    s = torch.cuda.current_stream(out.device).cuda_stream
    _lib.check(_lib.lib().ens_normals(int(seed), int(index_offset), int(n_traj), int(n_per),
                                      _TORCH_DT[dtype], _ptr(out), ctypes.c_void_p(s)))
    return out


def ensemble_moments(out, status=None, *, layout="rowmajor", slot=-1, stream=None):
    """Per-component moments of an ensemble's solution through ens_moments: a float64 tensor
    [2D + 1] on out's device = (mean_0..mean_{D-1}, M2_0..M2_{D-1}, n), M2 = sum of squared
    deviations from the mean, at save slot `slot` (negative: from the end) of a solve output
    (row-major [N, D] / [N, S, D], SoA [D, N] / [S, D, N]), over the trajectories with status 0
    (all without a status tensor)."""
    if not (out.is_cuda and out.is_contiguous()):
        raise ValueError("out must be a contiguous CUDA tensor")
    if layout == "rowmajor":
        N, S, D = (out.shape[0], 1, out.shape[1]) if out.dim() == 2 else tuple(out.shape)
    else:
        S, D, N = (1, out.shape[0], out.shape[1]) if out.dim() == 2 else tuple(out.shape)
    slot = slot + S if slot < 0 else slot
    if status is not None and (status.dtype != torch.int8 or status.numel() != N):
        raise ValueError("status must be an int8 tensor of N entries")
    res = torch.empty(2 * D + 1, dtype=torch.float64, device=out.device)
    scratch = torch.empty(_lib.MOMENTS_BLOCKS * (2 * D + 1), dtype=torch.float64,
                          device=out.device)
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream(out.device).cuda_stream
    _lib.check(_lib.lib().ens_moments(
        int(N), int(D), _TORCH_DT[out.dtype], _lib.LAYOUT[layout], int(S), int(slot),
        _ptr(out), _ptr(status) if status is not None else None, _ptr(scratch), _ptr(res),
        ctypes.c_void_p(s)))
    return res


def gather_moments(moments, group=None):
    """The exchange step of a sharded ensemble: every rank's ensemble_moments result, stacked
    in rank order ([world, 2D + 1]; [1, 2D + 1] without a process group).  An all-gather over
    torch.distributed (NCCL wants the tensor on the GPU, gloo on the CPU)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        parts = [torch.empty_like(moments) for _ in range(dist.get_world_size(group))]
        dist.all_gather(parts, moments.contiguous(), group=group)
        return torch.stack(parts)
    return moments.reshape(1, -1)


def merge_moments(parts):
    """Merge per-group (mean, M2, n) rows [k, 2D + 1] into the union's (n, mean [D],
    variance [D]) with ens_moments_combine (the pairwise update, in row order); the unbiased
    variance is M2 / (n - 1).  Raises ValueError when fewer than two trajectories count."""
    p = np.ascontiguousarray(parts.detach().cpu().numpy() if torch.is_tensor(parts) else parts,
                             dtype=np.float64)
    p = p.reshape(p.shape[0] if p.ndim > 1 else 1, -1)
    D = (p.shape[1] - 1) // 2
    res = np.empty(2 * D + 1)
    dp = ctypes.POINTER(ctypes.c_double)
    _lib.check(_lib.lib().ens_moments_combine(int(p.shape[0]), int(D), p.ctypes.data_as(dp),
                                              res.ctypes.data_as(dp)))
    n = res[2 * D]
    if n < 2:
        raise ValueError("the ensemble variance needs at least two counted trajectories "
                         "(n = %d)" % int(n))
    return n, res[:D], res[D:2 * D] / (n - 1)


def combine_moments(moments, group=None):
    """Gather every rank's ensemble_moments (gather_moments) and merge them (merge_moments):
    (n, mean [D], unbiased variance [D]) of the whole sharded ensemble."""
    return merge_moments(gather_moments(moments, group))


class EnsembleBatch:
    """Several sub-problems solved by one call (one CUDA graph launch with graph=True).
    fused=True runs them in one persistent kernel (ENS_BATCH_FUSED: Lorenz FP32 adaptive
    Tsit5, Robertson FP32 Rosenbrock23, GBM FP32 Euler-Maruyama, at most one of each);
    autotune=True times the concurrent, serial and (where allowed) fused forms and keeps the
    fastest.

    items: list of dicts with keys rhs ("lorenz" / "robertson" / "gbm" / "crn"), params, u0, tspan
    (CUDA tensors, one dtype per item), alg, layout (default "soa") and any ens_solve option
    (dt, abstol, reltol, dt0, maxiters, saveat, seed, index_offset, ...).  Outputs are
    allocated here: ``batch.outputs[i] = (out, status, stats)``.
    """

    def __init__(self, items, *, graph=True, autotune=False, serial=False, fused=False,
                 want_stats=True, stream=None):
        if not items or len(items) > _lib.BATCH_MAX_ITEMS:
            raise ValueError("1 .. %d items" % _lib.BATCH_MAX_ITEMS)
        arr = (_lib.BatchItem * len(items))()
        self.outputs, self._keep = [], []
        dev = None
        for k, it in enumerate(items):
            rhs_id = _lib.RHS[it["rhs"]]
            D, P = _lib.DIMS[rhs_id]
            params, u0, tspan = it["params"], it["u0"], it["tspan"]
            layout = it.get("layout", "soa")
            if params.dtype not in _TORCH_DT or u0.dtype != params.dtype or \
                    tspan.dtype != params.dtype:
                raise ValueError("item %d: params, u0, tspan must share float32/float64" % k)
            N = params.shape[0] if layout == "rowmajor" else params.shape[-1]
            saveat = it.get("saveat")
            saved = saveat is not None and len(saveat) > 0
            S = len(saveat) if saved else 1
            shp = ((N, P), (N, D), (N, 2)) if layout == "rowmajor" else ((P, N), (D, N), (2, N))
            for name, t, sh in zip(("params", "u0", "tspan"), (params, u0, tspan), shp):
                if tuple(t.shape) != sh or not t.is_contiguous() or not t.is_cuda:
                    raise ValueError("item %d: %s must be a contiguous CUDA tensor %s"
                                     % (k, name, sh))
            dev = params.device
            so = ((N, S, D) if saved else (N, D)) if layout == "rowmajor" else \
                ((S, D, N) if saved else (D, N))
            out = torch.empty(so, dtype=params.dtype, device=dev)
            status = torch.empty(N, dtype=torch.int8, device=dev)
            stats = torch.empty((3, N), dtype=torch.int32, device=dev) if want_stats else None
            kw = {k2: v for k2, v in it.items()
                  if k2 not in ("rhs", "params", "u0", "tspan", "alg", "layout")}
            o, keep = make_opts(it.get("alg", "tsit5"), _TORCH_DT[params.dtype], layout, **kw)
            arr[k].rhs_id = rhs_id
            arr[k].N = N
            arr[k].params, arr[k].u0, arr[k].tspan = (params.data_ptr(), u0.data_ptr(),
                                                      tspan.data_ptr())
            arr[k].out = out.data_ptr()
            arr[k].status = status.data_ptr()
            arr[k].stats = stats.data_ptr() if stats is not None else None
            arr[k].opts = o
            self.outputs.append((out, status, stats))
            self._keep.append((params, u0, tspan, keep))
        flags = (_lib.BATCH_GRAPH if graph else 0) | (_lib.BATCH_AUTOTUNE if autotune else 0) | \
            (_lib.BATCH_SERIAL if serial else 0) | (_lib.BATCH_FUSED if fused else 0)
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
        h = ctypes.c_void_p()
        _lib.check(_lib.lib().ens_batch_create(ctypes.byref(h), arr, len(items), flags,
                                               ctypes.c_void_p(s)))
        self._h = h
        self._items = arr
        self.device = dev

    def run(self, stream=None):
        s = torch.cuda.current_stream(self.device).cuda_stream if stream is None \
            else stream.cuda_stream
        _lib.check(_lib.lib().ens_batch_run(self._h, ctypes.c_void_p(s)))
        return self.outputs

    def info(self):
        res = []
        for k in range(len(self.outputs)):
            inf = _lib.BatchItemInfo()
            _lib.check(_lib.lib().ens_batch_info(self._h, k, ctypes.byref(inf)))
            res.append({"schedule": inf.schedule, "block": inf.block, "tpt": inf.tpt,
                        "blocks_per_sm": inf.blocks_per_sm,
                        "tuned_ms": inf.tuned_ms, "launch_position": inf.launch_position,
                        "graph": bool(inf.graph), "serial": bool(inf.serial),
                        "graph_ms_concurrent": inf.graph_ms_concurrent,
                        "graph_ms_serial": inf.graph_ms_serial,
                        "graph_ms_fused": inf.graph_ms_fused, "fused": bool(inf.fused),
                        "lane_slots": int(inf.lane_slots)})
        return res

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().ens_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
