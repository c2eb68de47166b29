"""Host-side checks of the C ABI that need no GPU: libens.so builds, loads and exports every
entry point include/*.h declares; argument validation fails before touching the device; the
product package does not reach the oracle."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ens_\w+)\s*\(", txt, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_2304_06835_gb300 import build
    build.build()
    from paper_2304_06835_gb300 import _lib
    return _lib.lib()


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("ens_create", "ens_destroy", "ens_solve", "ens_solve_host", "ens_last_error",
              "ens_philox4x32_10", "ens_normals", "ens_opts_default"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    for n in declared_symbols():
        assert hasattr(L, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2304_06835_gb300 import _lib
    assert set(declared_symbols()) <= set(_lib.SIGNATURES)


def test_validation_without_device(L):
    import ctypes
    from paper_2304_06835_gb300 import _lib
    o = _lib.EnsOpts()
    L.ens_opts_default(ctypes.byref(o))
    assert o.alg == 2 and o.maxiters == 1000000 and o.layout == 1
    rc = L.ens_solve(None, 10, None, None, None, ctypes.byref(o), None, None, None, None)
    assert rc == _lib.ENS_EINVAL
    assert b"handle" in L.ens_last_error()
    assert L.ens_philox4x32_10(1, 0, -1, 1, None, None) == _lib.ENS_EINVAL
    assert L.ens_normals(1, 0, 4, 4, 7, None, None) == _lib.ENS_EINVAL
    h = ctypes.c_void_p()
    assert L.ens_create(ctypes.byref(h), 99, 3, 3) == _lib.ENS_EINVAL
    assert L.ens_create(ctypes.byref(h), 1, 2, 3) == _lib.ENS_EINVAL
    # ens_moments(N, D, dtype, layout, S, slot, out, status, scratch, sums, stream)
    p = ctypes.c_void_p(16)  # never dereferenced: every call below fails validation first
    for args in ((-1, 3, 0, 0, 1, 0, p, None, p, p),   # N < 0
                 (4, 0, 0, 0, 1, 0, p, None, p, p),    # D < 1
                 (4, 3, 0, 0, 2, 2, p, None, p, p),    # slot >= S
                 (4, 3, 0, 0, 2, -1, p, None, p, p),   # slot < 0
                 (4, 3, 5, 0, 1, 0, p, None, p, p),    # dtype
                 (4, 3, 0, 7, 1, 0, p, None, p, p),    # layout
                 (4, 3, 0, 0, 1, 0, None, None, p, p),  # out
                 (4, 3, 0, 0, 1, 0, p, None, None, p),  # scratch
                 (4, 3, 0, 0, 1, 0, p, None, p, None)):  # sums
        assert L.ens_moments(*args, None) == _lib.ENS_EINVAL, args
    # ens_moments_combine(n_parts, D, parts, result): host arithmetic, runs without a GPU
    dp = ctypes.POINTER(ctypes.c_double)
    parts = np.array([[1.0, 2.0, 3.0], [4.0, 0.0, 1.0]])  # D = 1: (mean, M2, n) per row
    res = np.empty(3)
    assert L.ens_moments_combine(2, 1, parts.ctypes.data_as(dp), res.ctypes.data_as(dp)) == 0
    np.testing.assert_allclose(res, [1.75, 2.0 + 0.0 + 9.0 * 3.0 * 1.0 / 4.0, 4.0], rtol=1e-15)
    assert L.ens_moments_combine(0, 1, parts.ctypes.data_as(dp), res.ctypes.data_as(dp)) == 1
    assert L.ens_moments_combine(2, 1, None, res.ctypes.data_as(dp)) == 1


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2304_06835_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if not os.path.isfile(path) or not path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            continue
        txt = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), path
        assert "ens_oracle" not in txt and "liboracle" not in txt, path


def test_oracle_shares_no_source_with_cuda_path():
    txt = open(os.path.join(ROOT, "oracle", "ens_oracle.cpp")).read()
    assert "#include \"" not in txt  # only system headers
