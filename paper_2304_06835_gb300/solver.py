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
              schedule="auto", block=0, tpt=0, refill_min=0, order="auto"):
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
    return o, keep


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class EnsembleSolver:
    """One solver handle for one right-hand side ("lorenz", "robertson" or "gbm")."""

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
              schedule="auto", block=0, tpt=0, refill_min=0, order="auto", want_status=True,
              want_stats=False, out=None, status=None, stats=None, stream=None):
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
                            saveat, seed, index_offset, schedule, block, tpt, refill_min, order)
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
        _lib.check(_lib.lib().ens_solve(self._h, N, _ptr(params), _ptr(u0), _ptr(tspan),
                                        ctypes.byref(o), _ptr(out), _ptr(status), _ptr(stats),
                                        ctypes.c_void_p(s)))
        del keep
        return out, status, stats

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
