"""Pins of the oracle's weak second-order stochastic Runge-Kutta step (GPUSIEA, Sec. 5.2.2: weak
order 2, diagonal noise), taken as the improved-Euler-type scheme of the paper's SRK family
(Sec. 3.3) with fit term R:

    Ybar = X + a h + b dW,  Y+- = X + a h +- b sqrt(h),
    X1 = X + (a(X) + a(Ybar)) h/2 + (b(Y+) + b(Y-) + 2 b(X)) dW/4 + (b(Y+) - b(Y-)) (dW^2 - h)/(4 sqrt h).

* The scheme has weak order 2: by Milstein's theorem it suffices that the first five moments
  of the one-step increment X1 - x agree with those of the exact solution to O(h^3).  Checked
  symbolically for a generic scalar SDE dX = a(X) dt + b(X) dW: the exact increment moments
  come from the generator L = a d/dx + (b^2/2) d^2/dx^2 (E (X_h - x)^k = sum_{m<=2} h^m/m!
  L^m (y - x)^k at y = x), the scheme's from Taylor expansions of a and b and the Gaussian
  moments of dW.  Removing the fit term, or halving the drift average, breaks the check.
* On GBM (a = mu X, b = sigma X) the scheme reduces by hand to
      X1 = X [1 + mu h + mu^2 h^2 / 2 + sigma dW (1 + mu h) + sigma^2 (dW^2 - h) / 2],
  and the oracle's step equals that for any normal; hence its exact discrete moments
      E X_n = X0 m1^n,  m1 = 1 + mu h + mu^2 h^2 / 2,
      E X_n^2 = X0^2 m2^n,  m2 = m1^2 + sigma^2 h (1 + mu h)^2 + sigma^4 h^2 / 2,
  which the oracle's Monte Carlo means meet within 4 standard errors, and whose distance
  from the continuous moments X0 e^(mu t), X0^2 e^((2 mu + sigma^2) t) falls like h^2.
* Streams: step k of trajectory i uses normal k of the trajectory's Philox stream (as
  Euler-Maruyama): a path rebuilt from oracle.normals and the GBM closed form equals the
  oracle's solve.
"""
import numpy as np
import pytest
import sympy as sp

import oracle


class _Trunc:
    """Polynomial in s = sqrt(h) and Z with sympy coefficients, truncated below s^6 (terms of
    order h^3 and above never enter the weak order 2 conditions)."""
    N = 6

    def __init__(self, terms=None):
        self.t = {k: v for k, v in (terms or {}).items() if k[0] < self.N and v != 0}

    def __add__(self, o):
        o = o if isinstance(o, _Trunc) else _Trunc({(0, 0): o})
        r = dict(self.t)
        for k, v in o.t.items():
            r[k] = sp.expand(r.get(k, 0) + v)
        return _Trunc(r)

    def __sub__(self, o):
        return self + o * (-1)

    def __mul__(self, o):
        if not isinstance(o, _Trunc):
            return _Trunc({k: sp.expand(v * o) for k, v in self.t.items()})
        r = {}
        for (p1, z1), v1 in self.t.items():
            for (p2, z2), v2 in o.t.items():
                if p1 + p2 < self.N:
                    k = (p1 + p2, z1 + z2)
                    r[k] = r.get(k, 0) + v1 * v2
        return _Trunc({k: sp.expand(v) for k, v in r.items()})

    def shift(self, q):  # times s^q (q may be -1 when every term has a factor s)
        assert all(k[0] + q >= 0 for k in self.t)
        return _Trunc({(k[0] + q, k[1]): v for k, v in self.t.items()})

    def expect(self):  # E over Z ~ N(0,1): E Z^n = (n-1)!! (n even), 0 (n odd)
        r = {}
        for (ps, pz), v in self.t.items():
            if pz % 2 == 0:
                r[ps] = r.get(ps, 0) + v * (sp.factorial2(pz - 1) if pz else 1)
        return {k: sp.expand(v) for k, v in r.items()}


def _scheme_moments(a, b, order=5, fit=True, drift_half=True):
    """E (X1 - x)^k (k = 1..5) of the scheme for generic a, b, as {power of s: coefficient}:
    a[i], b[i] are the i-th derivatives at x; dW = s Z."""
    one = _Trunc({(0, 0): 1})
    s1, h, dW = _Trunc({(1, 0): 1}), _Trunc({(2, 0): 1}), _Trunc({(1, 1): 1})

    def taylor(c, d):
        out, p = one * c[0], one
        for i in range(1, order + 1):
            p = p * d
            out = out + p * (c[i] / sp.factorial(i))
        return out
    a0, b0 = a[0], b[0]
    abar = taylor(a, h * a0 + dW * b0)
    bp = taylor(b, h * a0 + s1 * b0)
    bm = taylor(b, h * a0 - s1 * b0)
    w = sp.Rational(1, 2) if drift_half else sp.Rational(1, 4)
    dX = (abar + a0) * h * w + (bp + bm + 2 * b0) * dW * sp.Rational(1, 4)
    if fit:  # (b(Y+) - b(Y-)) (dW^2 - h) / (4 s): every term of b(Y+) - b(Y-) has a factor s
        dX = dX + (bp - bm).shift(-1) * (dW * dW - h) * sp.Rational(1, 4)
    out, pw = [], one
    for _ in range(5):
        pw = pw * dX
        out.append(pw.expect())
    return out


def _exact_moments(a, b):
    """E (X_h - x)^k (k = 1..5) of the exact solution to O(h^3), as {power of s: coefficient}."""
    y, x = sp.symbols("y x")
    A, B = sp.Function("A")(y), sp.Function("B")(y)
    L = lambda g: A * sp.diff(g, y) + B ** 2 / 2 * sp.diff(g, y, 2)
    out = []
    for k in range(1, 6):
        g = (y - x) ** k
        g1 = L(g)
        g2 = L(g1)
        terms = {0: g, 2: g1, 4: g2 / 2}
        res = {}
        for q, e in terms.items():
            e = e.subs(y, x).doit()
            rep = {}
            for i in range(6, 0, -1):
                rep[sp.Derivative(sp.Function("A")(x), (x, i))] = a[i]
                rep[sp.Derivative(sp.Function("B")(x), (x, i))] = b[i]
            e = e.subs(rep).subs({sp.Function("A")(x): a[0], sp.Function("B")(x): b[0]})
            e = sp.expand(e)
            if e != 0:
                res[q] = e
        out.append(res)
    return out


def _same(m1, m2):
    keys = set(m1) | set(m2)
    return all(sp.expand(m1.get(q, 0) - m2.get(q, 0)) == 0 for q in keys)


@pytest.fixture(scope="module")
def symbols():
    a = sp.symbols("a0:7")
    b = sp.symbols("b0:7")
    return a, b, _exact_moments(a, b)


def test_scheme_has_weak_order_two(symbols):
    a, b, exact = symbols
    got = _scheme_moments(a, b)
    for k, (g, e) in enumerate(zip(got, exact), start=1):
        assert _same(g, e), k


@pytest.mark.parametrize("variant", [dict(fit=False), dict(drift_half=False)])
def test_weak_order_check_detects_a_broken_scheme(symbols, variant):
    a, b, exact = symbols
    got = _scheme_moments(a, b, **variant)
    assert not all(_same(g, e) for g, e in zip(got, exact))


def gbm_closed_form(x, mu, sig, h, z):
    dW = np.sqrt(h) * z
    return x * (1 + mu * h + mu * mu * h * h / 2 + sig * dW * (1 + mu * h)
                + sig * sig * (dW * dW - h) / 2)


def test_gbm_step_equals_the_hand_reduction():
    rng = np.random.default_rng(1)
    for _ in range(200):
        x, mu, sig = rng.uniform(0.2, 3), rng.uniform(-1, 1), rng.uniform(0.05, 0.8)
        h, z = 10 ** rng.uniform(-4, -0.5), rng.normal()
        got = oracle.step("gbm", "siea", [x], [mu, sig], 0.0, h, z)[0][0]
        ref = gbm_closed_form(x, mu, sig, h, z)
        assert abs(got - ref) <= 1e-13 * max(abs(ref), 1.0), (got, ref)
    # zero noise: Heun's method on u' = mu u
    got = oracle.step("gbm", "siea", [1.0], [0.3, 0.0], 0.0, 0.1, 0.7)[0][0]
    assert abs(got - (1 + 0.03 + 0.03 ** 2 / 2)) < 1e-15


def test_gbm_exact_discrete_moments_and_weak_order():
    M, mu, sig, h, n = 1 << 16, 0.4, 0.5, 0.02, 50
    P = np.tile([mu, sig], (M, 1))
    out, st, _ = oracle.solve("gbm", "siea", P, np.ones((M, 1)), np.tile([0.0, n * h], (M, 1)),
                              dt=h, seed=2024)
    assert np.all(st == 0)
    x = out[:, 0]
    m1 = 1 + mu * h + mu * mu * h * h / 2
    m2 = m1 * m1 + sig * sig * h * (1 + mu * h) ** 2 + sig ** 4 * h * h / 2
    assert abs(x.mean() - m1 ** n) < 4 * x.std() / np.sqrt(M)
    assert abs((x * x).mean() - m2 ** n) < 4 * (x * x).std() / np.sqrt(M)
    # the discrete moments approach the continuous ones like h^2 (weak order 2)
    T = 1.0
    e1, e2 = [], []
    for hh in (0.1, 0.05, 0.025):
        nn = int(round(T / hh))
        q1 = 1 + mu * hh + mu * mu * hh * hh / 2
        q2 = q1 * q1 + sig * sig * hh * (1 + mu * hh) ** 2 + sig ** 4 * hh * hh / 2
        e1.append(abs(q1 ** nn - np.exp(mu * T)))
        e2.append(abs(q2 ** nn - np.exp((2 * mu + sig * sig) * T)))
    for e in (e1, e2):
        slopes = np.diff(np.log(e)) / np.log(0.5)
        assert np.all(np.abs(slopes - 2) < 0.15), slopes


def test_stream_by_step_index():
    P = np.array([[0.3, 0.4], [-0.2, 0.3]])
    U = np.array([[1.0], [2.0]])
    T = np.array([[0.0, 0.05], [0.0, 0.05]])
    h = 0.01
    out, _, _ = oracle.solve("gbm", "siea", P, U, T, dt=h, seed=99, index_offset=7)
    for i in range(2):
        z = oracle.normals(99, 7 + i, 5, fp64=True)
        x = U[i, 0]
        for k in range(5):
            x = gbm_closed_form(x, P[i, 0], P[i, 1], h, z[k])
        assert abs(out[i, 0] - x) <= 1e-14 * abs(x)
