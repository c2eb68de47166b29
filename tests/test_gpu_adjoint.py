"""GPU parity of the discrete adjoint (ens_adjoint_forward / ens_adjoint) against the oracle's
exact gradient of the same discrete map (forward-mode tangents through every stage), plus
checkpoint invariance, the autograd wrapper and central differences of the GPU forward solve.

Tolerances: FP64 gradient, per trajectory, max |g - g_ref| / max(max |g_ref|, 1) <= 1e-10
(two exact gradients of one map that differ only in rounding order); FP32 <= 2e-4 against
the FP64 tangents on the float-rounded inputs (float rounding of ~1e3 steps, each step's
Jacobian product of norm O(1)).  Checkpoint intervals change no arithmetic: bit-identical.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def dev(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().double().numpy()


def normwise(g, ref):
    g = g.reshape(g.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.abs(g - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1.0)


@pytest.fixture(scope="module")
def S():
    from paper_2304_06835_gb300 import EnsembleSolver
    return {k: EnsembleSolver(k) for k in ("lorenz", "robertson", "gbm")}


def lorenz_case(N, seed, t1=1.0, uneven=False):
    P, U, T = workloads.lorenz_random(N, seed=seed, t1=t1)
    U = U + np.random.default_rng(seed + 1).normal(0, 1, U.shape)
    if uneven:
        T[:, 1] = np.random.default_rng(seed + 2).uniform(0.0, t1, N)
        T[: max(1, N // 50), 1] = 0.0       # tf == t0: zero steps
    G = workloads.adjoint_targets(N, seed=seed)
    return P, U, T, G


@pytest.mark.parametrize("alg", ["tsit5_fixed", "rk4"])
@pytest.mark.parametrize("N", [1, 33, 1000])
def test_adjoint_fp64_matches_oracle_tangents(S, alg, N):
    P, U, T, G = lorenz_case(N, seed=N + 3, uneven=N > 1)
    dt = 1.3e-2                               # ragged last step on most spans
    gp_ref, gu_ref, uf_ref = oracle.fixed_grad("lorenz", alg, P, U, T, dt, G)
    s = S["lorenz"]
    out, ckpt, st, ms = s.adjoint_forward(dev(P), dev(U), dev(T), alg, dt=dt, checkpoint_every=7)
    assert normwise(host(out), uf_ref).max() <= 1e-12
    assert int(st.abs().sum()) == 0
    gp, gu = s.adjoint(dev(P), dev(U), dev(T), dev(G), alg, dt=dt, checkpoint_every=7, ckpt=ckpt)
    assert normwise(host(gp), gp_ref).max() <= 1e-10
    assert normwise(host(gu), gu_ref).max() <= 1e-10
    zero = T[:, 1] == T[:, 0]
    if zero.any():  # no steps: dL/du0 = dL/du(tf), dL/dp = 0
        np.testing.assert_array_equal(host(gu)[zero], G[zero])
        assert np.all(host(gp)[zero] == 0)


def test_adjoint_fp32_close_to_fp64_tangents(S):
    P, U, T, G = lorenz_case(512, seed=11)
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    P, U, T, G = f(P), f(U), f(T), f(G)
    dt = 1e-2
    gp_ref, gu_ref, _ = oracle.fixed_grad("lorenz", "tsit5_fixed", P, U, T, dt, G)
    d32 = lambda a: dev(a, torch.float32)
    gp, gu = S["lorenz"].adjoint(d32(P), d32(U), d32(T), d32(G), "tsit5_fixed", dt=dt)
    assert normwise(host(gp), gp_ref).max() <= 2e-4
    assert normwise(host(gu), gu_ref).max() <= 2e-4


def test_adjoint_gbm_linear_closed_form(S):
    """u' = mu u, Tsit5: du(1)/du0 = R(h mu)^n and du(1)/dmu = n h R'(h mu) R^{n-1} u0."""
    c, A, b, _ = oracle.tsit5_tableau()
    mu = np.linspace(-0.5, 0.5, 64)
    P = np.stack([mu, np.full(64, 0.3)], axis=1)
    U = np.full((64, 1), 1.3)
    T = np.tile([0.0, 1.0], (64, 1))
    h, n = 0.01, 100
    R = lambda z: 1 + z * b @ np.linalg.solve(np.eye(7) - z * A, np.ones(7))
    gp, gu = S["gbm"].adjoint(dev(P), dev(U), dev(T), dev(np.ones((64, 1))), "tsit5_fixed", dt=h)
    gp, gu = host(gp), host(gu)
    for i, m in enumerate(mu):
        z = h * m
        Rp = (R(z + 1e-7) - R(z - 1e-7)) / 2e-7
        assert abs(gu[i, 0] - R(z) ** n) <= 1e-13 * max(1, abs(R(z) ** n))
        assert abs(gp[i, 0] - n * h * Rp * R(z) ** (n - 1) * 1.3) <= 1e-7
        assert gp[i, 1] == 0.0


def test_checkpoint_interval_and_layout_change_no_arithmetic(S):
    P, U, T, G = lorenz_case(777, seed=21, uneven=True)
    s = S["lorenz"]
    dt = 1e-2
    ref = None
    for every in (1, 7, 64, 1000):
        for with_ckpt in (True, False):
            ck = None
            if with_ckpt:
                _, ck, _, _ = s.adjoint_forward(dev(P), dev(U), dev(T), dt=dt,
                                                checkpoint_every=every)
            gp, gu = s.adjoint(dev(P), dev(U), dev(T), dev(G), dt=dt, checkpoint_every=every,
                               ckpt=ck)
            cur = np.concatenate([host(gp), host(gu)], axis=1)
            if ref is None:
                ref = cur
            else:
                np.testing.assert_array_equal(cur, ref)
    gp, gu = s.adjoint(dev(P.T), dev(U.T), dev(T.T), dev(G.T), dt=dt, layout="soa")
    np.testing.assert_array_equal(np.concatenate([host(gp).T, host(gu).T], axis=1), ref)


def test_max_steps_exceeded_reports_status(S):
    P, U, T, G = lorenz_case(40, seed=5)
    T[::2, 1] = 0.5
    s = S["lorenz"]
    out, ck, st, _ = s.adjoint_forward(dev(P), dev(U), dev(T), dt=1e-2, max_steps=60,
                                       checkpoint_every=16)
    st = st.cpu().numpy()
    assert np.all(st[::2] == 0) and np.all(st[1::2] == 1)  # 50 steps fit, 100 do not
    assert np.all(np.isnan(host(out)[1::2]))
    gp, gu = s.adjoint(dev(P), dev(U), dev(T), dev(G), dt=1e-2, max_steps=60,
                       checkpoint_every=16, ckpt=ck)
    assert np.all(np.isnan(host(gp)[1::2])) and np.all(np.isfinite(host(gp)[::2]))


def test_autograd_matches_adjoint_and_central_differences(S):
    from paper_2304_06835_gb300 import solve_fixed
    P, U, T, _ = lorenz_case(16, seed=31)
    tgt = dev(workloads.adjoint_targets(16, seed=31))
    s = S["lorenz"]
    dt = 1e-2
    p = dev(P).requires_grad_(True)
    u = dev(U).requires_grad_(True)
    Td = dev(T)
    loss = ((solve_fixed(s, p, u, Td, dt=dt) - tgt) ** 2).sum()
    loss.backward()
    out, _, _ = s.solve(dev(P), dev(U), Td, alg="tsit5_fixed", dt=dt)
    gp_ref, gu_ref = s.adjoint(dev(P), dev(U), Td, 2 * (out - tgt), dt=dt)
    np.testing.assert_array_equal(host(p.grad), host(gp_ref))
    np.testing.assert_array_equal(host(u.grad), host(gu_ref))

    def L(Pv, Uv):
        o, _, _ = s.solve(dev(Pv), dev(Uv), Td, alg="tsit5_fixed", dt=dt)
        return host(((o - tgt) ** 2).sum(dim=1))

    hh = 1e-6
    for m in range(3):
        e = np.zeros_like(P)
        e[:, m] = hh
        fd = (L(P + e, U) - L(P - e, U)) / (2 * hh)
        np.testing.assert_allclose(host(p.grad)[:, m], fd, rtol=1e-6, atol=1e-6)
        e = np.zeros_like(U)
        e[:, m] = hh
        fd = (L(P, U + e) - L(P, U - e)) / (2 * hh)
        np.testing.assert_allclose(host(u.grad)[:, m], fd, rtol=1e-6, atol=1e-6)


def test_adjoint_full_size_sampled():
    """The gradient workload at its full size in the launch configuration the bench times:
    Lorenz N = 65,536, [0,1], Tsit5 dt = 1e-3 (1000 steps), FP64, checkpoints every 64 steps,
    loss sum_i ||u_i(1) - target_i||^2; 512 sampled trajectories against the oracle."""
    from paper_2304_06835_gb300 import EnsembleSolver
    N = 65536
    P, U, T = workloads.lorenz_random(N, seed=5, t1=1.0)
    tgt = workloads.adjoint_targets(N, seed=5)
    s = EnsembleSolver("lorenz")
    Pd, Ud, Td = dev(P.T), dev(U.T), dev(T.T)
    out, ck, st, ms = s.adjoint_forward(Pd, Ud, Td, dt=1e-3, layout="soa", checkpoint_every=64)
    assert ms == 1000 and int(st.abs().sum()) == 0
    G = 2 * (out - dev(tgt.T))
    gp, gu = s.adjoint(Pd, Ud, Td, G, dt=1e-3, layout="soa", checkpoint_every=64, ckpt=ck)
    idx = np.random.default_rng(0).choice(N, 512, replace=False)
    gp_ref, gu_ref, uf = oracle.fixed_grad("lorenz", "tsit5_fixed", P[idx], U[idx], T[idx], 1e-3,
                                           host(G).T[idx])
    assert normwise(host(out).T[idx], uf).max() <= 1e-12
    assert normwise(host(gp).T[idx], gp_ref).max() <= 1e-10
    assert normwise(host(gu).T[idx], gu_ref).max() <= 1e-10
    assert np.all(np.isfinite(host(gp))) and np.all(np.isfinite(host(gu)))


def test_adjoint_rejects_bad_arguments(S):
    from paper_2304_06835_gb300 import EnsError
    P, U, T, G = lorenz_case(4, seed=1)
    s = S["lorenz"]
    with pytest.raises(EnsError):
        s.adjoint(dev(P), dev(U), dev(T), dev(G), "tsit5", dt=1e-2)        # adaptive
    with pytest.raises(EnsError):
        s.adjoint(dev(P), dev(U), dev(T), dev(G), dt=0.0, max_steps=10)
    with pytest.raises(EnsError):
        s.adjoint(dev(P), dev(U), dev(T), dev(G), dt=1e-2, checkpoint_every=0)
