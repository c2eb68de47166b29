"""CPU oracle for the ensemble ODE/SDE solver -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs
may import this package.  The product package never imports it and shares no code with it.

The arithmetic lives in ``ens_oracle.cpp`` (plain C++, FP64, with an FP32 mode), built on demand
into ``liboracle.so`` next to this file; ``mlp.py`` holds the NumPy oracle of the surrogate
network.  This module only marshals NumPy arrays into the C functions.

Identifiers (the same numbers as the public C-ABI, by documentation):
  rhs:  1 Lorenz (D=3, P=3: sigma, rho, beta), 2 Robertson (D=3, P=3: k1, k2, k3),
        3 geometric Brownian motion (D=1, P=2: mu, sigma; 1 Wiener process),
        4 sigma-factor CRN (D=4: [sigma], A1, A2, A3; P=6: S, D, tau, nu0, n, eta;
          8 Wiener processes; Euler-Maruyama only),
        5 bouncing ball (D=2: x, v; P=2: g, e; the event x = 0 from above sets v <- -e v;
          adaptive Tsit5 only),
        6 Oregonator (D=3, P=3: k1, k2, k3), 7 HIRES (D=8, P=12: its distinct rate constants),
        8 POLLU (D=20, P=25: k1..k25) -- the paper's stiff test models
  alg:  1 Tsit5 fixed, 2 Tsit5 adaptive, 3 RK4, 4 Rosenbrock23, 5 Euler-Maruyama,
        6 Rodas4, 7 Rodas5P (stiffly accurate Rosenbrock 4(3) and 5(4)),
        8 SIEA (weak order 2 stochastic Runge-Kutta, diagonal noise: GBM)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ens_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

RHS = {"lorenz": 1, "robertson": 2, "gbm": 3, "crn": 4, "ball": 5, "orego": 6, "hires": 7,
       "pollu": 8}
ALG = {"tsit5_fixed": 1, "tsit5": 2, "rk4": 3, "ros23": 4, "em": 5, "rodas4": 6, "rodas5p": 7,
       "siea": 8}
DIMS = {1: (3, 3), 2: (3, 3), 3: (1, 2), 4: (4, 6), 5: (2, 2), 6: (3, 3), 7: (8, 12),
        8: (20, 25)}
NOISE = {1: 0, 2: 0, 3: 1, 4: 8, 5: 0, 6: 0, 7: 0, 8: 0}  # Wiener processes per model
STATUS = {"ok": 0, "maxiters": 1, "dt_min": 2, "nonfinite": 3}


def _compile(src: str, target: str) -> None:
    tmp = target + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
           "-o", tmp, src]
    subprocess.check_call(cmd)
    os.replace(tmp, target)


def build(force: bool = False) -> str:
    """Compile liboracle.so with the host compiler (no FMA contraction, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        _compile(_SRC, _LIB)
    return _LIB


def source() -> str:
    """The oracle's C++ source text (tests plant mistakes in copies of it)."""
    with open(_SRC) as f:
        return f.read()


class variant:
    """Context manager: compile a modified copy of the oracle's source into `workdir` and
    route every call of this module to it until the block ends.  Used by tests that plant
    a mistake in the oracle and check that a pin detects it."""

    def __init__(self, text: str, workdir: str):
        self.text, self.workdir = text, workdir

    def __enter__(self):
        global _lib
        src = os.path.join(self.workdir, "ens_oracle_variant.cpp")
        so = os.path.join(self.workdir, "liboracle_variant.so")
        with open(src, "w") as f:
            f.write(self.text)
        _compile(src, so)
        lib()  # the regular library first, so that it is restored afterwards
        with _lock:
            self._saved = _lib
            _lib = _bind(ctypes.CDLL(so))
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self._saved
        return False


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _bind(L):
    """Declare the C signatures of the oracle's entry points on a loaded library."""
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_solve.restype = ctypes.c_int
    L.oracle_solve.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
        dp, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
        ctypes.c_longlong, dp, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_longlong,
        dp, ctypes.POINTER(ctypes.c_byte), ctypes.POINTER(ctypes.c_longlong), ctypes.c_int,
        ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_longlong)]
    L.oracle_solve_steps.restype = ctypes.c_int
    L.oracle_solve_steps.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, dp, dp, dp,
        ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_longlong,
        ctypes.c_double, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_byte),
        ctypes.POINTER(ctypes.c_longlong), dp, dp, ctypes.POINTER(ctypes.c_longlong),
        ctypes.c_int]
    L.oracle_pollu_reaction_sum.restype = None
    L.oracle_pollu_reaction_sum.argtypes = [dp, dp, dp]
    L.oracle_tsit5_dense.restype = None
    L.oracle_tsit5_dense.argtypes = [dp]
    L.oracle_step.restype = ctypes.c_int
    L.oracle_step.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double, dp, dp]
    L.oracle_rosenbrock_tableau.restype = ctypes.c_int
    L.oracle_rosenbrock_tableau.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
    L.oracle_tsit5_tableau.restype = None
    L.oracle_tsit5_tableau.argtypes = [dp, dp, dp, dp]
    L.oracle_rhs.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp]
    L.oracle_jac.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp, dp]
    L.oracle_diffusion.restype = ctypes.c_int
    L.oracle_diffusion.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp]
    L.oracle_em_step.restype = ctypes.c_int
    L.oracle_em_step.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                                 dp, dp]
    L.oracle_lu_solve.argtypes = [ctypes.c_int, dp, dp, dp]
    u32p = ctypes.POINTER(ctypes.c_uint32)
    L.oracle_philox4x32_10.restype = None
    L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.oracle_normals.restype = None
    L.oracle_normals.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.c_longlong,
                                 ctypes.c_int, dp]
    L.oracle_tsit5_fixed_grad.restype = ctypes.c_int
    L.oracle_tsit5_fixed_grad.argtypes = [ctypes.c_int, ctypes.c_longlong, dp, dp, dp,
                                          ctypes.c_double, dp, dp, dp, dp, ctypes.c_int]
    L.oracle_fixed_grad.restype = ctypes.c_int
    L.oracle_fixed_grad.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, dp, dp,
                                    dp, ctypes.c_double, dp, dp, dp, dp, ctypes.c_int]
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def solve(rhs, alg, params, u0, tspan, *, dt=0.0, abstol=1e-6, reltol=1e-3, dt0=0.0,
          maxiters=1_000_000, saveat=None, seed=0, index_offset=0, precision="f64",
          nthreads=None, dense=False, dtmax=0.0, want_events=False):
    """Solve an ensemble.  params [N,P], u0 [N,D], tspan [N,2] (row-major, float64).

    precision "f32" runs the same algorithms in float arithmetic on the given (already
    float-representable) inputs; "f64_f32stream" is FP64 arithmetic driven by the FP32 normal
    stream (4 normals per Philox call).  dense=True (adaptive Tsit5 with saveat): the steps
    run to tf without being cut at save times, which take the dense output (oracle/dense.py).
    dtmax > 0 caps the adaptive step; want_events=True appends the events handled per
    trajectory [N] to the result (bouncing ball).  Returns (out [N,S,D] or [N,D], status [N], stats [N,3]).
    """
    rhs_id = RHS[rhs] if isinstance(rhs, str) else int(rhs)
    alg_id = ALG[alg] if isinstance(alg, str) else int(alg)
    D, P = DIMS[rhs_id]
    params = _f64(params).reshape(-1, P)
    N = params.shape[0]
    u0 = _f64(u0).reshape(N, D)
    tspan = _f64(tspan).reshape(N, 2)
    sv = None if saveat is None else _f64(saveat).reshape(-1)
    S = 1 if sv is None or sv.size == 0 else sv.size
    out = np.empty((N, S, D), np.float64)
    status = np.empty(N, np.int8)
    stats = np.empty((N, 3), np.int64)
    events = np.zeros(N, np.int64)
    nt = default_threads() if nthreads is None else int(nthreads)
    rc = lib().oracle_solve(
        rhs_id, alg_id, {"f64": 0, "f32": 1, "f64_f32stream": 2}[precision], 0, N, _dp(params), _dp(u0), _dp(tspan),
        float(dt), float(abstol), float(reltol), float(dt0), int(maxiters),
        _dp(sv) if sv is not None and sv.size else None, 0 if sv is None else int(sv.size),
        int(seed), int(index_offset), _dp(out),
        status.ctypes.data_as(ctypes.POINTER(ctypes.c_byte)),
        stats.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), nt, 1 if dense else 0,
        float(dtmax), events.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    if rc != 0:
        raise ValueError("oracle_solve rejected its arguments")
    if sv is None or sv.size == 0:
        out = out[:, 0, :]
    if want_events:
        return out, status, stats, events
    return out, status, stats


def solve_steps(rhs, alg, params, u0, tspan, cap, *, abstol=1e-6, reltol=1e-3, dt0=0.0,
                maxiters=1_000_000, dtmax=0.0, precision="f64", nthreads=None):
    """Every accepted step of an adaptive solve: returns (t [N, cap], u [N, cap, D],
    n [N] = accepted steps + 1 (entry 0 is the initial state; entries past n are NaN; n may
    exceed cap), out [N, D], status [N], stats [N, 3])."""
    rhs_id = RHS[rhs] if isinstance(rhs, str) else int(rhs)
    alg_id = ALG[alg] if isinstance(alg, str) else int(alg)
    D, P = DIMS[rhs_id]
    params = _f64(params).reshape(-1, P)
    N = params.shape[0]
    u0 = _f64(u0).reshape(N, D)
    tspan = _f64(tspan).reshape(N, 2)
    out = np.empty((N, D))
    status = np.empty(N, np.int8)
    stats = np.empty((N, 3), np.int64)
    rt = np.empty((N, cap))
    ru = np.empty((N, cap, D))
    rn = np.empty(N, np.int64)
    nt = default_threads() if nthreads is None else int(nthreads)
    ll = ctypes.POINTER(ctypes.c_longlong)
    rc = lib().oracle_solve_steps(
        rhs_id, alg_id, {"f64": 0, "f32": 1}[precision], N, _dp(params), _dp(u0), _dp(tspan),
        float(abstol), float(reltol), float(dt0), int(maxiters), float(dtmax), int(cap),
        _dp(out), status.ctypes.data_as(ctypes.POINTER(ctypes.c_byte)), stats.ctypes.data_as(ll),
        _dp(rt), _dp(ru), rn.ctypes.data_as(ll), nt)
    if rc != 0:
        raise ValueError("oracle_solve_steps rejected its arguments")
    return rt, ru, rn, out, status, stats


def step(rhs, alg, u, p, t, h, z=0.0):
    """One step of a method; returns (u_new, err)."""
    rhs_id = RHS[rhs] if isinstance(rhs, str) else int(rhs)
    alg_id = ALG[alg] if isinstance(alg, str) else int(alg)
    D, _ = DIMS[rhs_id]
    u = _f64(u)
    p = _f64(p)
    unew = np.empty(D)
    err = np.empty(D)
    if lib().oracle_step(rhs_id, alg_id, _dp(u), _dp(p), float(t), float(h), float(z), _dp(unew),
                         _dp(err)) != 0:
        raise ValueError("bad step arguments")
    return unew, err


def tsit5_dense():
    """The typed dense-output coefficients r [7, 4] of the C++ oracle."""
    r = np.empty(28)
    lib().oracle_tsit5_dense(_dp(r))
    return r.reshape(7, 4)


def tsit5_tableau():
    c = np.empty(7)
    A = np.empty((7, 7))
    b = np.empty(7)
    bh = np.empty(7)
    lib().oracle_tsit5_tableau(_dp(c), _dp(A), _dp(b), _dp(bh))
    return c, A, b, bh


def rosenbrock_tableau(alg):
    """Standard-form coefficients of Rodas4 / Rodas5P as the oracle steps them:
    (gamma, alpha [s,s], Gamma [s,s] with gamma on the diagonal, b [s], bhat [s])."""
    alg_id = ALG[alg] if isinstance(alg, str) else int(alg)
    g = ctypes.c_double()
    A = np.empty(64)
    G = np.empty(64)
    b = np.empty(8)
    bh = np.empty(8)
    s = lib().oracle_rosenbrock_tableau(alg_id, ctypes.byref(g), _dp(A), _dp(G), _dp(b), _dp(bh))
    if s < 0:
        raise ValueError("not a Rodas method")
    return g.value, A.reshape(8, 8)[:s, :s], G.reshape(8, 8)[:s, :s], b[:s], bh[:s]


def rhs_eval(rhs, u, p, t=0.0):
    rhs_id = RHS[rhs] if isinstance(rhs, str) else int(rhs)
    D, _ = DIMS[rhs_id]
    du = np.empty(D)
    lib().oracle_rhs(rhs_id, _dp(_f64(u)), _dp(_f64(p)), float(t), _dp(du))
    return du


def diffusion(rhs, u, p, t=0.0):
    """Diffusion matrix G [D, Mw] of an SDE model (column m multiplies dW_{m+1})."""
    rhs_id = RHS[rhs] if isinstance(rhs, str) else int(rhs)
    D, _ = DIMS[rhs_id]
    G = np.empty((D, NOISE[rhs_id]))
    if lib().oracle_diffusion(rhs_id, _dp(_f64(u)), _dp(_f64(p)), float(t), _dp(G)) != 0:
        raise ValueError("not an SDE model")
    return G


def em_step(rhs, u, p, t, h, z):
    """One Euler-Maruyama step with the given normals z [Mw]."""
    rhs_id = RHS[rhs] if isinstance(rhs, str) else int(rhs)
    D, _ = DIMS[rhs_id]
    z = _f64(z).reshape(-1)
    if z.size != NOISE[rhs_id]:
        raise ValueError("need one normal per Wiener process")
    unew = np.empty(D)
    if lib().oracle_em_step(rhs_id, _dp(_f64(u)), _dp(_f64(p)), float(t), float(h), _dp(z),
                            _dp(unew)) != 0:
        raise ValueError("not an SDE model")
    return unew


def jac_u(rhs, u, p, t=0.0):
    """df/du [D, D] (every model with a Jacobian, the stiff test models included)."""
    rhs_id = RHS[rhs] if isinstance(rhs, str) else int(rhs)
    D, _ = DIMS[rhs_id]
    Ju = np.empty((D, D))
    if lib().oracle_jac(rhs_id, _dp(_f64(u)), _dp(_f64(p)), float(t), _dp(Ju), None) != 0:
        raise ValueError("model without a Jacobian")
    return Ju


def pollu_reaction_sum(y, k):
    """POLLU's right-hand side formed as the sum over its 25 mass-action reactions."""
    dy = np.empty(20)
    lib().oracle_pollu_reaction_sum(_dp(_f64(y)), _dp(_f64(k)), _dp(dy))
    return dy


def jacobians(rhs, u, p, t=0.0):
    rhs_id = RHS[rhs] if isinstance(rhs, str) else int(rhs)
    D, P = DIMS[rhs_id]
    Ju = np.empty((D, D))
    Jp = np.empty((D, P))
    lib().oracle_jac(rhs_id, _dp(_f64(u)), _dp(_f64(p)), float(t), _dp(Ju), _dp(Jp))
    return Ju, Jp


def lu_solve(W, b):
    W = _f64(W)
    D = W.shape[0]
    x = np.empty(D)
    lib().oracle_lu_solve(D, _dp(W), _dp(_f64(b)), _dp(x))
    return x


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib().oracle_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p),
                               out.ctypes.data_as(u32p))
    return out


def normals(seed, traj, n, fp64=False):
    out = np.empty(int(n))
    lib().oracle_normals(int(seed), int(traj), int(n), 1 if fp64 else 0, _dp(out))
    return out


def tsit5_fixed_grad(rhs, params, u0, tspan, dt, grad_out, nthreads=None):
    """Exact gradient of the fixed-step Tsit5 map by forward tangents.

    Returns (grad_p [N,P], grad_u0 [N,D], u_final [N,D])."""
    return fixed_grad(rhs, "tsit5_fixed", params, u0, tspan, dt, grad_out, nthreads)


def fixed_grad(rhs, alg, params, u0, tspan, dt, grad_out, nthreads=None):
    """Exact gradient of a fixed-step explicit RK map ("tsit5_fixed" or "rk4") by forward
    tangents: grad_out [N,D] = dL/du(tf).  Returns (grad_p [N,P], grad_u0 [N,D], u_final [N,D])."""
    rhs_id = RHS[rhs] if isinstance(rhs, str) else int(rhs)
    alg_id = ALG[alg] if isinstance(alg, str) else int(alg)
    D, P = DIMS[rhs_id]
    params = _f64(params).reshape(-1, P)
    N = params.shape[0]
    u0 = _f64(u0).reshape(N, D)
    tspan = _f64(tspan).reshape(N, 2)
    go = _f64(grad_out).reshape(N, D)
    gp = np.empty((N, P))
    gu = np.empty((N, D))
    uf = np.empty((N, D))
    nt = default_threads() if nthreads is None else int(nthreads)
    rc = lib().oracle_fixed_grad(rhs_id, alg_id, N, _dp(params), _dp(u0), _dp(tspan), float(dt),
                                 _dp(go), _dp(gp), _dp(gu), _dp(uf), nt)
    if rc != 0:
        raise ValueError("bad arguments")
    return gp, gu, uf
