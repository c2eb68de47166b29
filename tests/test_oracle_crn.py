"""Pins of the oracle's sigma-factor CRN SDE and of its Euler-Maruyama with several Wiener
processes (Appendix, CRN model; Sec. 3.3 Euler-Maruyama) to facts fixed outside the oracle:

* drift values at points where the Hill term is computed by hand (integer and fractional
  exponents, a negative amount that the max(., 0) reading clamps);
* the Chemical Langevin structure of the noise: each Wiener process drives one species, and
  G G^T equals the sum over reactions of propensity x stoichiometry^2 (production and decay of
  [sigma], the three conversion steps of the A chain);
* with S = 0 the drift is linear and the Euler-Maruyama mean and covariance obey exact
  recursions (mean: the Euler map; covariance: B C B^T + h E[G G^T], affine in the mean while
  no amount reaches zero) -- checked by Monte Carlo over the oracle's own Philox streams;
* with eta = 0 and S = 0, the path equals the matrix-power solution of the Euler recursion;
* the stream reading: step k uses normals k*8 .. k*8+7 of the trajectory's stream.
"""
import numpy as np
import pytest

import oracle
import workloads

NOISE = 8


def test_crn_drift_hand_values():
    # (S sigma)^n = (2*1)^2 = 4, (D A3)^n = (1*1)^2 = 1, H = 4/6; tau = 0.5
    u = [1.0, 0.5, 0.25, 1.0]
    p = [2.0, 1.0, 0.5, 0.1, 2.0, 0.05]
    np.testing.assert_allclose(oracle.rhs_eval("crn", u, p),
                               [0.1 + 4.0 / 6.0 - 1.0, 1.0, 0.5, -1.5], rtol=1e-15, atol=1e-15)
    # fractional exponent: (8*0.5)^1.5 = 8, (0.5*2)^1.5 = 1, H = 0.8; tau = 2
    u = [0.5, 0.0, 0.0, 2.0]
    p = [8.0, 0.5, 2.0, 0.05, 1.5, 0.0]
    np.testing.assert_allclose(oracle.rhs_eval("crn", u, p), [0.05 + 0.8 - 0.5, 0.25, 0.0, -1.0],
                               rtol=1e-15, atol=1e-15)
    # S and D enter on different species: swapping them changes H from 4/6 to 1/6
    u = [1.0, 0.5, 0.25, 1.0]
    p = [1.0, 2.0, 0.5, 0.1, 2.0, 0.05]
    assert oracle.rhs_eval("crn", u, p)[0] == pytest.approx(0.1 + 1.0 / 6.0 - 1.0, abs=1e-15)
    # a negative [sigma] clamps its Hill base at 0: H = 0
    u = [-0.3, 0.0, 0.0, 1.0]
    p = [5.0, 1.0, 1.0, 0.1, 2.5, 0.05]
    assert oracle.rhs_eval("crn", u, p)[0] == pytest.approx(0.1 + 0.3, abs=1e-15)


def _cle_diffusion(u, p, H):
    """G G^T of the Chemical Langevin equation: reactions (propensity, stoichiometry)
    0 -> sigma (nu0 + H, e0), sigma -> 0 (sigma, -e0), 0 -> A1 (sigma/tau, e1),
    A1 -> 0 (A1/tau, -e1), 0 -> A2 (A1/tau, e2), A2 -> 0 (A2/tau, -e2), 0 -> A3 (A2/tau, e3),
    A3 -> 0 (A3/tau, -e3); every Wiener process carries eta."""
    s, a1, a2, a3 = u
    tau, nu0, eta = p[2], p[3], p[5]
    return eta ** 2 * np.diag([nu0 + H + s, (s + a1) / tau, (a1 + a2) / tau, (a2 + a3) / tau])


def test_crn_noise_is_the_chemical_langevin_form():
    u = [1.0, 0.5, 0.25, 1.0]
    p = [2.0, 1.0, 0.5, 0.1, 2.0, 0.05]
    G = oracle.diffusion("crn", u, p)
    assert G.shape == (4, NOISE)
    # each Wiener process drives exactly one species: dW_{2j+1}, dW_{2j+2} act on species j
    for m in range(NOISE):
        rows = np.flatnonzero(G[:, m])
        assert list(rows) == [m // 2]
        assert (G[m // 2, m] > 0) == (m % 2 == 0)  # production +, decay -
    np.testing.assert_allclose(G @ G.T, _cle_diffusion(u, p, 4.0 / 6.0), rtol=1e-14, atol=1e-18)
    # negative amounts: the square-root arguments clamp at 0
    G = oracle.diffusion("crn", [-0.2, 0.3, -0.1, 0.4], p)
    assert G[0, 1] == 0.0 and G[1, 2] == 0.0 and G[2, 5] == 0.0 and G[3, 6] == 0.0
    assert np.all(np.isfinite(G))


def _linear_chain(p, h):
    """S = 0: drift A u + b (exact, H = 0); Euler map u -> B u + h b."""
    tau, nu0 = p[2], p[3]
    A = np.array([[-1.0, 0, 0, 0], [1 / tau, -1 / tau, 0, 0], [0, 1 / tau, -1 / tau, 0],
                  [0, 0, 1 / tau, -1 / tau]])
    b = np.array([nu0, 0.0, 0.0, 0.0])
    return np.eye(4) + h * A, h * b


def test_crn_zero_noise_linear_chain_matches_matrix_powers():
    h, K = 0.1, 100
    p = np.array([0.0, 3.0, 0.7, 0.15, 2.0, 0.0])
    u0 = np.array([1.0, 0.2, 0.6, 0.0])
    B, c = _linear_chain(p, h)
    want = np.linalg.matrix_power(B, K) @ u0 + sum(np.linalg.matrix_power(B, i) @ c
                                                   for i in range(K))
    out, st, stats = oracle.solve("crn", "em", p[None], u0[None], [[0.0, K * h]], dt=h, seed=3)
    assert st[0] == 0 and stats[0, 0] == K
    np.testing.assert_allclose(out[0], want, rtol=1e-13, atol=1e-15)


def test_crn_em_mean_and_covariance_recursions():
    """Monte Carlo over 20000 oracle streams; 6 standard errors (the inputs keep every amount
    far from zero, so no clamp acts and E[G G^T] is the affine function of the mean)."""
    h, K, N = 0.1, 60, 20000
    p = np.array([0.0, 1.0, 2.0, 0.2, 2.0, 0.05])
    u0 = np.array([1.0, 1.0, 0.5, 0.8])
    B, c = _linear_chain(p, h)
    m, C = u0.copy(), np.zeros((4, 4))
    checkpoints = {}
    for k in range(1, K + 1):
        C = B @ C @ B.T + h * _cle_diffusion(m, p, 0.0)
        m = B @ m + c
        if k in (1, 10, K):
            checkpoints[k] = (m.copy(), C.copy())
    P = np.repeat(p[None], N, 0)
    U = np.repeat(u0[None], N, 0)
    for k, (mk, Ck) in checkpoints.items():
        T = np.tile([0.0, k * h], (N, 1))
        out, st, _ = oracle.solve("crn", "em", P, U, T, dt=h, seed=11)
        assert np.all(st == 0) and out.min() > 0.0
        se_m = np.sqrt(np.diag(Ck) / N)
        assert np.all(np.abs(out.mean(0) - mk) < 6 * se_m), (k, out.mean(0), mk)
        Ce = np.cov(out.T)
        se_c = np.sqrt((np.outer(np.diag(Ck), np.diag(Ck)) + Ck ** 2) / N)
        assert np.all(np.abs(Ce - Ck) < 6 * se_c), (k, Ce, Ck)


def test_crn_stream_reading_step_k_uses_normals_8k_to_8k_plus_7():
    p, u0, _ = workloads.crn_random(3, seed=1)
    h, seed = 0.1, 77
    for traj in range(3):
        z = oracle.normals(seed, traj, 3 * NOISE, fp64=True)  # the FP64 solve draws 2 per call
        u = u0[traj]
        for k in range(3):
            hk = h if k < 2 else 3 * h - 2 * h  # the last step ends exactly at tf
            u = oracle.em_step("crn", u, p[traj], k * h, hk, z[k * NOISE:(k + 1) * NOISE])
        out, _, _ = oracle.solve("crn", "em", p, u0, np.tile([0.0, 3 * h], (3, 1)), dt=h,
                                 seed=seed)
        np.testing.assert_array_equal(out[traj], u)


def test_crn_rejects_methods_without_noise_or_jacobian():
    p, u0, T = workloads.crn_random(2, seed=1, t1=1.0)
    for alg in ("tsit5", "rk4", "ros23"):
        with pytest.raises(ValueError):
            oracle.solve("crn", alg, p, u0, T, dt=0.1)


def test_crn_paper_workload_f32_mode_close_to_f64():
    p, u0, T = workloads.crn_random(64, seed=2, t1=100.0)
    p32, u32, T32 = (a.astype(np.float32).astype(np.float64) for a in (p, u0, T))
    o64, s64, _ = oracle.solve("crn", "em", p32, u32, T32, dt=0.1, seed=5,
                               precision="f64_f32stream")
    o32, s32, _ = oracle.solve("crn", "em", p32, u32, T32, dt=0.1, seed=5, precision="f32")
    assert np.all(s64 == 0) and np.all(s32 == 0)
    np.testing.assert_allclose(o32, o64, rtol=1e-3, atol=1e-4)
