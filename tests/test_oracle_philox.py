"""Pins of the oracle's counter-based generator (Philox4x32-10, Salmon et al. SC'11) and of the
normal draws that drive Euler-Maruyama (Sec. 3.3: dW ~ N(0, dt); Sec. 6.7: the seed supplied to
the PRNG)."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_known_answers(ctr, key, expect):
    out = oracle.philox4x32_10(ctr, key)
    assert [int(x) for x in out] == expect


def test_normals_fp32_distribution():
    z = np.concatenate([oracle.normals(1234, tr, 4000, fp64=False) for tr in range(50)])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 6 * np.sqrt(2 / z.size)


def test_normals_fp64_distribution():
    z = np.concatenate([oracle.normals(99, tr, 4000, fp64=True) for tr in range(50)])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 4 / np.sqrt(z.size)


def test_streams_independent():
    a = oracle.normals(7, 0, 20000)
    b = oracle.normals(7, 1, 20000)
    c = oracle.normals(8, 0, 20000)
    for x, y in ((a, b), (a, c)):
        r = np.corrcoef(x, y)[0, 1]
        assert abs(r) < 4 / np.sqrt(x.size)
    # lag-1 autocorrelation inside a stream
    r1 = np.corrcoef(a[:-1], a[1:])[0, 1]
    assert abs(r1) < 4 / np.sqrt(a.size)


def test_uniform_mapping_is_box_muller_of_philox_words():
    """The FP32 stream's normals 0 and 1 come from the uniforms of words 0 and 1 of the first
    Philox call; check the Box-Muller identity z0^2 + z1^2 = -2 ln u0 on those words."""
    seed, tr = 0x1234_5678_9ABC, 5
    x = oracle.philox4x32_10([0, 0, tr, 0], [seed & 0xFFFFFFFF, seed >> 32])
    u0 = ((int(x[0]) >> 9) + 0.5) * 2.0**-23
    z = oracle.normals(seed, tr, 4)
    assert abs(z[0] ** 2 + z[1] ** 2 - (-2 * np.log(u0))) < 1e-12
    u2 = ((int(x[2]) >> 9) + 0.5) * 2.0**-23
    assert abs(z[2] ** 2 + z[3] ** 2 - (-2 * np.log(u2))) < 1e-12
