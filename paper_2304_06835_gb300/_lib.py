"""ctypes binding of libens.so: argument marshalling only (see include/ens.h).

Every computation runs in the library's CUDA kernels.  If libens.so is missing this module
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libens.so")

ENS_OK, ENS_EINVAL, ENS_ENOTSUP, ENS_ECUDA, ENS_ENOMEM = 0, 1, 2, 3, 4
RHS = {"lorenz": 1, "robertson": 2, "gbm": 3, "crn": 4, "ball": 5, "orego": 6, "hires": 7,
       "pollu": 8}
DIMS = {1: (3, 3), 2: (3, 3), 3: (1, 2), 4: (4, 6), 5: (2, 2), 6: (3, 3), 7: (8, 12), 8: (20, 25)}
NOISE = {1: 0, 2: 0, 3: 1, 4: 8, 5: 0, 6: 0, 7: 0, 8: 0}  # Wiener processes per model
ALG = {"tsit5_fixed": 1, "tsit5": 2, "rk4": 3, "ros23": 4, "em": 5, "rodas4": 6, "rodas5p": 7,
       "siea": 8}
F32, F64 = 0, 1
LAYOUT = {"rowmajor": 0, "soa": 1}
MOMENTS_BLOCKS = 608  # ENS_MOMENTS_BLOCKS
SCHED = {"auto": 0, "direct": 1, "persistent": 2}
ORDER = {"auto": 0, "index": 1, "cost": 2}
MAX_SAVE = 256
STATUS = {0: "ok", 1: "maxiters", 2: "dt_min", 3: "nonfinite"}


class EnsOpts(ctypes.Structure):
    _fields_ = [
        ("alg", ctypes.c_int), ("dtype", ctypes.c_int), ("layout", ctypes.c_int),
        ("dt", ctypes.c_double), ("abstol", ctypes.c_double), ("reltol", ctypes.c_double),
        ("dt0", ctypes.c_double), ("maxiters", ctypes.c_longlong),
        ("saveat", ctypes.POINTER(ctypes.c_double)), ("n_save", ctypes.c_int),
        ("seed", ctypes.c_ulonglong), ("index_offset", ctypes.c_longlong),
        ("schedule", ctypes.c_int), ("block", ctypes.c_int), ("tpt", ctypes.c_int),
        ("refill_min", ctypes.c_int), ("order", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
        ("dense", ctypes.c_int), ("dtmax", ctypes.c_double), ("step_cap", ctypes.c_int),
        ("step_t", ctypes.c_void_p), ("step_n", ctypes.c_void_p),
        ("kernel_start", ctypes.c_void_p), ("kernel_stop", ctypes.c_void_p),
    ]


class BatchItem(ctypes.Structure):
    _fields_ = [
        ("rhs_id", ctypes.c_int), ("N", ctypes.c_longlong), ("params", ctypes.c_void_p),
        ("u0", ctypes.c_void_p), ("tspan", ctypes.c_void_p), ("out", ctypes.c_void_p),
        ("status", ctypes.c_void_p), ("stats", ctypes.c_void_p), ("opts", EnsOpts),
    ]


class BatchItemInfo(ctypes.Structure):
    _fields_ = [
        ("schedule", ctypes.c_int), ("block", ctypes.c_int), ("tpt", ctypes.c_int),
        ("blocks_per_sm", ctypes.c_int), ("tuned_ms", ctypes.c_float),
        ("launch_position", ctypes.c_int), ("graph", ctypes.c_int), ("serial", ctypes.c_int),
        ("graph_ms_concurrent", ctypes.c_float), ("graph_ms_serial", ctypes.c_float),
        ("graph_ms_fused", ctypes.c_float), ("fused", ctypes.c_int),
        ("lane_slots", ctypes.c_ulonglong),
    ]


BATCH_GRAPH, BATCH_AUTOTUNE, BATCH_SERIAL, BATCH_FUSED = 1, 2, 4, 8
BATCH_MAX_ITEMS = 16


class EnsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("ens error %d: %s" % (code, msg))
        self.code = code


_lock = threading.Lock()
_lib = None

_VP = ctypes.c_void_p
_LL = ctypes.c_longlong
_INT = ctypes.c_int
_ULL = ctypes.c_ulonglong

SIGNATURES = {
    "ens_opts_default": (None, [ctypes.POINTER(EnsOpts)]),
    "ens_create": (_INT, [ctypes.POINTER(_VP), _INT, _INT, _INT]),
    "ens_destroy": (_INT, [_VP]),
    "ens_solve": (_INT, [_VP, _LL, _VP, _VP, _VP, ctypes.POINTER(EnsOpts), _VP, _VP, _VP, _VP]),
    "ens_solve_host": (_INT, [_VP, _LL, _VP, _VP, _VP, ctypes.POINTER(EnsOpts), _VP, _VP, _VP,
                              _VP]),
    "ens_cost_keys": (_INT, [_VP, _LL, _VP, _VP, _VP, ctypes.POINTER(EnsOpts), _VP, _VP]),
    "ens_philox4x32_10": (_INT, [_ULL, _LL, _LL, _LL, _VP, _VP]),
    "ens_normals": (_INT, [_ULL, _LL, _LL, _LL, _INT, _VP, _VP]),
    "ens_moments": (_INT, [_LL, _INT, _INT, _INT, _INT, _INT, _VP, _VP, _VP, _VP, _VP]),
    "ens_moments_combine": (_INT, [_INT, _INT, _VP, _VP]),
    "ens_solve_noalloc": (_INT, [_INT, _LL, _VP, _VP, _VP, ctypes.POINTER(EnsOpts), _VP, _VP, _VP,
                                 _VP]),
    "ens_autotune": (_INT, [_VP, _LL, _VP, _VP, _VP, ctypes.POINTER(EnsOpts), _VP, _VP, _VP, _VP,
                            ctypes.POINTER(_INT), ctypes.POINTER(_INT), ctypes.POINTER(_INT),
                            ctypes.POINTER(ctypes.c_float)]),
    "ens_batch_create": (_INT, [ctypes.POINTER(_VP), ctypes.POINTER(BatchItem), _INT, _INT, _VP]),
    "ens_batch_run": (_INT, [_VP, _VP]),
    "ens_batch_info": (_INT, [_VP, _INT, ctypes.POINTER(BatchItemInfo)]),
    "ens_batch_destroy": (_INT, [_VP]),
    "ens_adjoint_ckpt_elems": (_LL, [_LL, _INT, _LL, _INT]),
    "ens_adjoint_forward": (_INT, [_VP, _LL, _VP, _VP, _VP, ctypes.POINTER(EnsOpts), _LL, _INT,
                                   _VP, _VP, _VP, _VP]),
    "ens_adjoint": (_INT, [_VP, _LL, _VP, _VP, _VP, ctypes.POINTER(EnsOpts), _LL, _INT, _VP, _VP,
                           _VP, _VP, _VP]),
    "ens_mlp_n_params": (_LL, []),
    "ens_mlp_create": (_INT, [ctypes.POINTER(_VP), _INT, _LL, ctypes.POINTER(ctypes.c_double), _ULL,
                              _VP]),
    "ens_mlp_destroy": (_INT, [_VP]),
    "ens_mlp_set_scaling": (_INT, [_VP, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), _VP]),
    "ens_mlp_params": (_INT, [_VP, _INT, _VP, _VP, _VP]),
    "ens_mlp_grad": (_INT, [_VP, _INT, _LL, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ens_mlp_adam": (_INT, [_VP, _INT, ctypes.c_float, _INT, _VP]),
    "ens_mlp_forward": (_INT, [_VP, _INT, _LL, _VP, _VP, _INT, _VP]),
    "ens_mlp_gate": (_INT, [_VP, _LL, _VP, _VP, ctypes.c_float, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                            ctypes.c_double, ctypes.c_double, _VP]),
    "ens_mlp_scatter": (_INT, [_LL, _VP, _VP, _VP, _VP]),
    "ens_mlp_check": (_INT, [_VP, _VP]),
    "ens_mlp_activation": (_INT, [_INT, _LL, _VP, _VP, _VP]),
    "ens_probe_fma": (_INT, [_INT, _LL, _INT, _INT, ctypes.POINTER(ctypes.c_double), _VP]),
    "ens_last_error": (ctypes.c_char_p, []),
}


def lib():
    """Load libens.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libens.so is not built: run paper_2304_06835_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(rc: int):
    if rc != ENS_OK:
        msg = lib().ens_last_error()
        raise EnsError(rc, msg.decode() if msg else "")


def exported_symbols():
    return [n for n in SIGNATURES if getattr(lib(), n, None) is not None]
