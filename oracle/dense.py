"""Continuous extension (dense output) of the Tsitouras 5(4) pair -- TEST INFRASTRUCTURE ONLY.

The paper saves adaptive solutions at requested times through the method's interpolant
(Sec. 5.1.1, solution storage; Sec. 5.2.1, GPUTsit5).  It does not print the interpolant's
coefficients.  This module defines one from the order conditions alone:

  u(t_n + theta h) = u_n + h sum_i b_i(theta) k_i,   b_i(theta) = sum_{q=1..4} r_iq theta^q,

with the seven stages k_i of the step (the 7th is f(u_{n+1}), FSAL), such that for every
theta in [0, 1]
  * the elementary-weight conditions of the 8 rooted trees of order <= 4 hold
    (sum_i b_i(theta) Phi_t,i = theta^r(t) / gamma(t)): the interpolant has order 4;
  * b_i(1) = b_i: it ends at u_{n+1};
  * b_i'(0) = [i = 1] and b_i'(1) = [i = 7]: its derivative is f at both ends (C1 across steps).
These leave a one-parameter family.  The member chosen minimises the 5th-order defect
  integral_0^1 sum_{t of order 5} (sum_i b_i(theta) Phi_t,i - theta^5 / gamma(t))^2 dtheta.
The computation runs in 40-digit arithmetic (mpmath); the tableau is the published one
(Tsitouras 2011), as decimal constants.

`derive()` returns r [7][4]; the C++ oracle types these values (`TS_DENSE`), and
tests/test_oracle_dense.py checks the typed constants against `derive()` and the
conditions above against the tableau.
"""
from __future__ import annotations

import mpmath as mp

TSIT5_C = ["0", "0.161", "0.327", "0.9", "0.9800255409045097", "1", "1"]
TSIT5_A = {1: ["0.161"], 2: ["-0.008480655492356989", "0.335480655492357"],
           3: ["2.897153057105493", "-6.359448489975075", "4.3622954328695815"],
           4: ["5.325864828439257", "-11.748883564062828", "7.4955393428898365",
               "-0.09249506636175525"],
           5: ["5.86145544294642", "-12.92096931784711", "8.159367898576159",
               "-0.071584973281401", "-0.028269050394068383"]}
TSIT5_B = ["0.09646076681806523", "0.01", "0.4798896504144996", "1.379008574103742",
           "-3.290069515436081", "2.324710524099774", "0"]
S = 7


def tableau():
    """(c, A, b) as mpmath numbers; stage 7 is the FSAL stage (a_7j = b_j, c_7 = 1)."""
    c = [mp.mpf(v) for v in TSIT5_C]
    A = [[mp.mpf(0)] * S for _ in range(S)]
    for i, row in TSIT5_A.items():
        for j, v in enumerate(row):
            A[i][j] = mp.mpf(v)
    b = [mp.mpf(v) for v in TSIT5_B]
    A[6] = list(b)
    return c, A, b


def elementary_weights(c, A):
    """Phi_t for the rooted trees of order <= 5: lists of (order, gamma, Phi[7])."""
    mv = lambda M, v: [mp.fsum(M[i][j] * v[j] for j in range(S)) for i in range(S)]
    ew = lambda u, v: [u[i] * v[i] for i in range(S)]
    pw = lambda v, k: [x ** k for x in v]
    one = [mp.mpf(1)] * S
    Ac, Ac2, Ac3 = mv(A, c), mv(A, pw(c, 2)), mv(A, pw(c, 3))
    AAc = mv(A, Ac)
    return [
        (1, 1, one), (2, 2, c),
        (3, 3, pw(c, 2)), (3, 6, Ac),
        (4, 4, pw(c, 3)), (4, 8, ew(c, Ac)), (4, 12, Ac2), (4, 24, AAc),
        (5, 5, pw(c, 4)), (5, 10, ew(pw(c, 2), Ac)), (5, 15, ew(c, Ac2)),
        (5, 30, ew(c, AAc)), (5, 20, ew(Ac, Ac)), (5, 20, Ac3), (5, 40, mv(A, ew(c, Ac))),
        (5, 60, mv(A, Ac2)), (5, 120, mv(A, AAc)),
    ]


def _constraints(c, A, b):
    rows, rhs = [], []
    for order, gamma, phi in elementary_weights(c, A):
        if order > 4:
            continue
        for q in range(1, 5):  # coefficient of theta^q
            r = [mp.mpf(0)] * 28
            for i in range(S):
                r[4 * i + q - 1] = phi[i]
            rows.append(r)
            rhs.append(mp.mpf(1) / gamma if q == order else mp.mpf(0))
    for i in range(S):
        r = [mp.mpf(0)] * 28
        for q in range(4):
            r[4 * i + q] = mp.mpf(1)
        rows.append(r), rhs.append(b[i])                               # b_i(1) = b_i
        r = [mp.mpf(0)] * 28
        r[4 * i] = mp.mpf(1)
        rows.append(r), rhs.append(mp.mpf(1 if i == 0 else 0))         # b_i'(0)
        r = [mp.mpf(0)] * 28
        for q in range(4):
            r[4 * i + q] = mp.mpf(q + 1)
        rows.append(r), rhs.append(mp.mpf(1 if i == S - 1 else 0))     # b_i'(1)
    return mp.matrix(rows), mp.matrix(rhs)


def defect5(x, c, A):
    """integral_0^1 of the summed squared 5th-order defects, exactly (polynomials in theta)."""
    tot = mp.mpf(0)
    for order, gamma, phi in elementary_weights(c, A):
        if order != 5:
            continue
        # defect(theta) = sum_{q=1..5} d_q theta^q
        d = [mp.fsum(x[4 * i + q] * phi[i] for i in range(S)) for q in range(4)]
        d.append(-mp.mpf(1) / gamma)
        tot += mp.fsum(d[p] * d[q] / (p + q + 3) for p in range(5) for q in range(5))
    return tot


_CACHE = {}


def family(dps: int = 40):
    """(x, null): the chosen member (28 mpmath numbers, stage-major) and the unit direction
    that the conditions leave free; evaluate inside mp.workdps(dps)."""
    with mp.workdps(dps):
        c, A, b = tableau()
        M, y = _constraints(c, A, b)
        U, sig, V = mp.svd_r(M)
        n = 28
        # every direction but the last is fixed by the conditions (rank 27; the tableau's
        # decimals satisfy the order-5 conditions only to ~1e-16, so the last singular value
        # is ~1e-17 rather than 0)
        x0 = mp.matrix(n, 1)
        for k in range(n - 1):
            coef = mp.fsum(U[j, k] * y[j] for j in range(M.rows)) / sig[k]
            for j in range(n):
                x0[j] += coef * V[k, j]
        null = mp.matrix([V[n - 1, j] for j in range(n)])
        f0, fp, fm = defect5(x0, c, A), defect5(x0 + null, c, A), defect5(x0 - null, c, A)
        a = -(fp - fm) / (2 * (fp + fm - 2 * f0))
        return x0 + a * null, null


def derive(dps: int = 40):
    """r [7][4] (floats) of the continuous extension defined above."""
    if dps in _CACHE:
        return _CACHE[dps]
    with mp.workdps(dps):
        x, _ = family(dps)
        r = [[float(x[4 * i + q]) for q in range(4)] for i in range(S)]
    r[0][0] = 1.0  # b_1'(0) = 1 and b_i'(0) = 0 hold exactly
    for i in range(1, S):
        r[i][0] = 0.0
    _CACHE[dps] = r
    return r


def weights(theta, r=None):
    """b_i(theta), i = 1..7 (Horner in theta)."""
    r = derive() if r is None else r
    return [theta * (ri[0] + theta * (ri[1] + theta * (ri[2] + theta * ri[3]))) for ri in r]


if __name__ == "__main__":
    for i, ri in enumerate(derive()):
        print("b%d: %s" % (i + 1, ", ".join(repr(v) for v in ri)))
