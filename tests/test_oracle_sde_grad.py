"""Pins of the oracle's Euler-Maruyama path (Sec. 3.3; GPUEM, Sec. 5.2.2; the linear asset-price
SDE, Appendix) and of its exact gradient of the fixed-step Tsit5 map (the discrete-adjoint
target; automatic differentiation through the solver is claimed in Sec. 6.5)."""
import numpy as np
import pytest

import oracle
import workloads


@pytest.mark.parametrize("fp", ["f32", "f64"])
def test_em_gbm_exact_discrete_moments(fp):
    """X_{k+1} = X_k (1 + mu h + sigma sqrt(h) Z_k) with iid N(0,1) Z gives
    E[X_n] = X0 (1+mu h)^n and E[X_n^2] = X0^2 ((1+mu h)^2 + sigma^2 h)^n exactly."""
    M = 1 << 16
    mu, sig, h, n = 0.4, 0.5, 1e-2, 100
    P = np.tile([mu, sig], (M, 1))
    U = np.ones((M, 1))
    T = np.tile([0.0, 1.0], (M, 1))
    out, st, stt = oracle.solve("gbm", "em", P, U, T, dt=h, seed=2023, precision=fp)
    assert np.all(st == 0) and np.all(stt[:, 0] == n)
    x = out[:, 0]
    m1 = (1 + mu * h) ** n
    m2 = ((1 + mu * h) ** 2 + sig * sig * h) ** n
    se1 = x.std() / np.sqrt(M)
    se2 = (x * x).std() / np.sqrt(M)
    assert abs(x.mean() - m1) < 4 * se1, (x.mean(), m1, se1)
    assert abs((x * x).mean() - m2) < 4 * se2, ((x * x).mean(), m2, se2)
    # weak error against the continuous GBM moments is O(h)
    assert abs(m1 - np.exp(mu)) < 0.02 and abs(m2 - np.exp(2 * mu + sig * sig)) < 0.1


def test_em_zero_noise_is_explicit_euler():
    P = np.array([[0.7, 0.0], [-0.3, 0.0]])
    out, _, _ = oracle.solve("gbm", "em", P, np.ones((2, 1)), np.tile([0.0, 1.0], (2, 1)),
                             dt=1e-3, seed=5)
    np.testing.assert_allclose(out[:, 0], (1 + P[:, 0] * 1e-3) ** 1000, rtol=1e-12)


def test_em_uses_stream_of_its_index():
    """Trajectory i's path is driven by stream index_offset + i (sharding-invariant)."""
    P, U, T = workloads.gbm_random(8, seed=1)
    full, _, _ = oracle.solve("gbm", "em", P, U, T, dt=1e-3, seed=77)
    part, _, _ = oracle.solve("gbm", "em", P[4:], U[4:], T[4:], dt=1e-3, seed=77, index_offset=4)
    np.testing.assert_array_equal(full[4:], part)
    # one step, by hand from the stream's first normal
    z0 = oracle.normals(77, 3, 1, fp64=True)[0]
    one, _, _ = oracle.solve("gbm", "em", P[3:4], U[3:4], [[0.0, 1e-3]], dt=1e-3, seed=77,
                             index_offset=3)
    mu, s = P[3]
    assert abs(one[0, 0] - (1 + mu * 1e-3 + s * np.sqrt(1e-3) * z0)) < 1e-15


@pytest.mark.parametrize("alg", ["tsit5_fixed", "rk4"])
def test_tangent_gradient_matches_central_differences(alg):
    P, U, T = workloads.lorenz_random(6, seed=5, t1=1.0)
    U = U + np.random.default_rng(3).normal(0, 1, U.shape)
    tgt = workloads.adjoint_targets(6)
    dt = 1e-2

    def loss(Pv, Uv):
        out, _, _ = oracle.solve("lorenz", alg, Pv, Uv, T, dt=dt)
        return ((out - tgt) ** 2).sum(axis=1)

    out, _, _ = oracle.solve("lorenz", alg, P, U, T, dt=dt)
    gp, gu, uf = oracle.fixed_grad("lorenz", alg, P, U, T, dt, 2 * (out - tgt))
    if alg == "tsit5_fixed":
        np.testing.assert_array_equal(uf, out)
    else:
        np.testing.assert_allclose(uf, out, rtol=1e-13, atol=1e-13)
    hh = 1e-6
    for m in range(3):
        e = np.zeros_like(P)
        e[:, m] = hh
        fd = (loss(P + e, U) - loss(P - e, U)) / (2 * hh)
        np.testing.assert_allclose(gp[:, m], fd, rtol=1e-6, atol=1e-6)
        e = np.zeros_like(U)
        e[:, m] = hh
        fd = (loss(P, U + e) - loss(P, U - e)) / (2 * hh)
        np.testing.assert_allclose(gu[:, m], fd, rtol=1e-6, atol=1e-6)


def test_tangent_gradient_linear_closed_form():
    """u' = mu u: u(1) = R(h mu)^n u0, so d u(1)/d u0 = R^n and d u(1)/d mu = n h R'(z) R^{n-1} u0."""
    c, A, b, _ = oracle.tsit5_tableau()
    mu, h, n, u0 = -0.8, 0.01, 100, 1.3
    z = h * mu
    s = A.shape[0]
    R = lambda zz: 1 + zz * b @ np.linalg.solve(np.eye(s) - zz * A, np.ones(s))
    dz = 1e-7
    Rp = (R(z + dz) - R(z - dz)) / (2 * dz)
    gp, gu, _ = oracle.tsit5_fixed_grad("gbm", [[mu, 0.2]], [[u0]], [[0.0, 1.0]], h, [[1.0]])
    assert abs(gu[0, 0] - R(z) ** n) < 1e-13
    assert abs(gp[0, 0] - n * h * Rp * R(z) ** (n - 1) * u0) < 1e-8
    assert gp[0, 1] == 0.0


def test_tangent_gradient_rk4_linear_closed_form():
    """RK4 on u' = mu u: R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, so du(1)/du0 = R^n and
    du(1)/dmu = n h R'(z) R^{n-1} u0 with R'(z) = 1 + z + z^2/2 + z^3/6."""
    mu, h, n, u0 = -0.8, 0.01, 100, 1.3
    z = h * mu
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    Rp = 1 + z + z * z / 2 + z ** 3 / 6
    gp, gu, _ = oracle.fixed_grad("gbm", "rk4", [[mu, 0.2]], [[u0]], [[0.0, 1.0]], h, [[1.0]])
    assert abs(gu[0, 0] - R ** n) < 1e-13
    assert abs(gp[0, 0] - n * h * Rp * R ** (n - 1) * u0) < 1e-12
