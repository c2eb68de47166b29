"""The Python binding's ctypes structures have the C layout of include/ens.h: a small C
program built with the host compiler prints sizeof / offsetof of every field, and each must
equal the ctypes one (a mismatch would pass garbage options without any error)."""
import ctypes
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(struct, fields):
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ens.h"', 'int main(void) {',
             '  printf("%%zu\\n", sizeof(%s));' % struct]
    lines += ['  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f) for f in fields]
    lines += ['  return 0;', '}']
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src,
                               "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("name", ["EnsOpts", "BatchItem", "BatchItemInfo"])
def test_ctypes_structs_match_the_header(name):
    from paper_2304_06835_gb300 import _lib
    cstruct = {"EnsOpts": "ens_opts", "BatchItem": "ens_batch_item",
               "BatchItemInfo": "ens_batch_item_info"}[name]
    S = getattr(_lib, name)
    fields = [f[0] for f in S._fields_]
    size, offs = _c_layout(cstruct, fields)
    assert ctypes.sizeof(S) == size
    assert [getattr(S, f).offset for f in fields] == offs
