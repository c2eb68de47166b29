"""Pins of the oracle's Tsit5 tableau to the Runge-Kutta order conditions (Sec. 3.1, tableau
{A, b, c}; Tsitouras 2011 5(4) pair named by GPUTsit5, Sec. 5.2.1).

The conditions are generated here from rooted trees (Butcher): for every rooted tree t with
|t| <= p nodes, b . Phi(t) = 1 / gamma(t).  A wrong digit in any coefficient, a transposed
entry or a misplaced weight breaks at least one condition.
"""
import itertools
from fractions import Fraction

import numpy as np

import oracle


def rooted_trees(n):
    """All rooted trees with n nodes, as sorted tuples of child subtrees (canonical form)."""
    if n == 1:
        return [()]
    out = set()
    # partitions of n-1 into child subtree sizes
    def parts(m, maxpart):
        if m == 0:
            yield []
            return
        for k in range(min(m, maxpart), 0, -1):
            for rest in parts(m - k, k):
                yield [k] + rest

    for sizes in parts(n - 1, n - 1):
        pools = [rooted_trees(s) for s in sizes]
        for combo in itertools.product(*pools):
            out.add(tuple(sorted(combo)))
    return sorted(out)


def gamma(t):
    n = 1 + sum(size(c) for c in t)
    g = n
    for c in t:
        g *= gamma(c)
    return g


def size(t):
    return 1 + sum(size(c) for c in t)


def phi(t, A):
    """Internal elementary weight vector: prod over children of A @ phi(child)."""
    v = np.ones(A.shape[0])
    for c in t:
        v = v * (A @ phi(c, A))
    return v


def test_tree_counts():
    # OEIS A000081: 1, 1, 2, 4, 9, 20
    assert [len(rooted_trees(n)) for n in range(1, 7)] == [1, 1, 2, 4, 9, 20]


def test_row_sums_and_fsal():
    c, A, b, bh = oracle.tsit5_tableau()
    np.testing.assert_allclose(A.sum(axis=1), c, atol=2e-15, rtol=0)
    np.testing.assert_array_equal(A[6, :6], b[:6])  # FSAL: last stage is f(u_{n+1})
    assert b[6] == 0.0
    assert np.all(np.triu(A) == 0)  # explicit
    assert c[0] == 0 and c[6] == 1.0


def test_order5_conditions_b():
    _, A, b, _ = oracle.tsit5_tableau()
    n_checked = 0
    for n in range(1, 6):
        for t in rooted_trees(n):
            lhs = float(b @ phi(t, A))
            assert abs(lhs - 1.0 / gamma(t)) < 2e-14, (t, lhs, 1.0 / gamma(t))
            n_checked += 1
    assert n_checked == 17


def test_order4_conditions_bhat_and_not_5():
    _, A, _, bh = oracle.tsit5_tableau()
    for n in range(1, 5):
        for t in rooted_trees(n):
            assert abs(float(bh @ phi(t, A)) - 1.0 / gamma(t)) < 2e-14, t
    # the embedded pair is genuinely of order 4: some order-5 condition fails for bhat
    worst = max(abs(float(bh @ phi(t, A)) - 1.0 / gamma(t)) for t in rooted_trees(5))
    assert worst > 1e-4


def test_b_not_order6():
    _, A, b, _ = oracle.tsit5_tableau()
    worst = max(abs(float(b @ phi(t, A)) - 1.0 / gamma(t)) for t in rooted_trees(6))
    assert worst > 1e-5


def test_stability_polynomial_rational():
    """R(z) = 1 + z b^T (I - zA)^{-1} 1 expanded with exact rationals of the printed
    coefficients: the first six Taylor coefficients are 1/k! up to the decimal rounding of
    the published coefficients."""
    _, A, b, _ = oracle.tsit5_tableau()
    Af = [[Fraction(x) for x in row] for row in A]
    bf = [Fraction(x) for x in b]
    # coefficient of z^k (k>=1) is b^T A^{k-1} 1
    v = [Fraction(1)] * 7
    coefs = [Fraction(1)]
    for k in range(1, 8):
        coefs.append(sum(bf[i] * v[i] for i in range(7)))
        v = [sum(Af[i][j] * v[j] for j in range(7)) for i in range(7)]
    import math
    for k in range(6):
        assert abs(float(coefs[k]) - 1.0 / math.factorial(k)) < 1e-14
    assert abs(float(coefs[6]) - 1.0 / 720) > 1e-6  # order exactly 5
    assert coefs[7] == 0  # b_7 = 0 and A strictly lower: degree 6
