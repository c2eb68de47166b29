"""GPU parity of the surrogate network's kernels (tcgen05 GEMMs with fused epilogues, loss,
bias sums, Adam, gate) against the NumPy oracle (oracle/mlp.py), which models the same bf16
rounding points in FP64 arithmetic.

Tolerances: forward, max |y - y_ref| <= 5e-3 max |y_ref| (FP32 accumulation order and erff
against FP64: a bf16 rounding of a hidden activation can land on the other side, a 2^-8
relative change of that activation); gradient, relative Frobenius error of every weight and
bias block <= 1e-2; Adam, 1e-6 relative (FP32 update arithmetic); gate flags exact away
from the threshold.
"""
import math

import numpy as np
import pytest
import torch

import workloads
from oracle import mlp

pytestmark = pytest.mark.gpu

BOX = workloads.surrogate_box()


def params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    layers = []
    for (wo, wi), (bo,) in mlp.param_shapes():
        layers.append((rng.normal(0, scale / math.sqrt(wi), (wo, wi)), rng.normal(0, 0.1, bo)))
    return mlp.flatten(layers).astype(np.float32).astype(np.float64)


def cuda32(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.fixture(scope="module")
def net():
    from paper_2304_06835_gb300 import SurrogateMLP
    m = SurrogateMLP(BOX, members=2, batch_max=4096, seed=3)
    yield m
    m.close()


def test_activation_within_published_error_bound():
    """The kernels' GELU and GELU' (erf by Abramowitz & Stegun 7.1.26, |error| <= 1.5e-7)
    against the exact erf forms in FP64."""
    import ctypes
    from paper_2304_06835_gb300 import _lib
    z = np.linspace(-12, 12, 200001).astype(np.float32)
    zd = cuda32(z)
    out = torch.empty_like(zd)
    for which, ref in ((0, mlp.gelu), (1, mlp.gelu_grad)):
        _lib.check(_lib.lib().ens_mlp_activation(which, z.size, ctypes.c_void_p(zd.data_ptr()),
                                                 ctypes.c_void_p(out.data_ptr()), None))
        r = ref(z.astype(np.float64))
        got = out.cpu().double().numpy()
        # 1.5e-7 from the approximation plus the approximate reciprocal and exponential
        # (2^-22 relative each), scaled by |z|/2 for gelu, plus float32 rounding
        bound = 5e-7 * (0.5 * np.abs(z) + 1) + 4e-7 * np.abs(r) + 1e-7
        assert np.all(np.abs(got - r) <= bound), np.max(np.abs(got - r) - bound)


@pytest.mark.parametrize("B", [1, 127, 1000, 4096])
def test_forward_matches_oracle(net, B):
    p = params(1)
    net.set_params(0, p)
    ym, ys = np.array([0.5, -1.0, 2.0]), np.array([2.0, 3.0, 4.0])
    net.set_scaling(ym, ys)
    x = workloads.surrogate_inputs(B, seed=B).astype(np.float32).astype(np.float64)
    ref = mlp.forward(p, x, BOX, ym, ys)
    y = net.forward(cuda32(x), member=0)[0].cpu().double().numpy()
    net.check()
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err <= 5e-3, err
    assert np.median(np.abs(y - ref)) <= 1e-3 * np.abs(ref).max()


def test_forward_all_members_and_chunking(net):
    """member = -1 returns every member; B beyond batch_max is processed in chunks."""
    p0, p1 = params(2), params(3)
    net.set_params(0, p0)
    net.set_params(1, p1)
    net.set_scaling(np.zeros(3), np.ones(3))
    x = workloads.surrogate_inputs(10000, seed=5).astype(np.float32).astype(np.float64)
    y = net.forward(cuda32(x)).cpu().double().numpy()
    assert y.shape == (2, 10000, 3)
    for k, p in enumerate((p0, p1)):
        ref = mlp.forward(p, x, BOX, np.zeros(3), np.ones(3))
        assert np.abs(y[k] - ref).max() <= 5e-3 * np.abs(ref).max()
    y0 = net.forward(cuda32(x[:4096]), member=0).cpu().double().numpy()[0]
    np.testing.assert_array_equal(y0, y[0, :4096])


@pytest.mark.parametrize("B", [1, 127, 128, 129, 1000, 4096, 10000])
def test_fused_forward_equals_layerwise(net, B):
    """The fused on-chip forward (all layers and members in one kernel) gives exactly the
    layer-by-layer result: same K order, same epilogue operations."""
    net.set_params(0, params(11))
    net.set_params(1, params(12))
    net.set_scaling(np.array([0.5, -1.0, 2.0]), np.array([2.0, 3.0, 4.0]))
    x = cuda32(workloads.surrogate_inputs(B, seed=40 + B))
    a = net.forward(x).cpu().numpy()
    b = net.forward(x, layerwise=True).cpu().numpy()
    net.check()
    np.testing.assert_array_equal(a, b)
    c = net.forward(x, member=1).cpu().numpy()[0]
    np.testing.assert_array_equal(c, b[1])


@pytest.mark.parametrize("B", [200, 4096])
def test_gradient_matches_oracle(net, B):
    p = params(4)
    net.set_params(1, p)
    ym, ys = np.array([0.1, 0.2, 0.3]), np.array([5.0, 6.0, 7.0])
    net.set_scaling(ym, ys)
    x = workloads.surrogate_inputs(B, seed=10 + B).astype(np.float32).astype(np.float64)
    y = np.random.default_rng(B).normal(0, 5, (B, 3)).astype(np.float32).astype(np.float64)
    loss_ref, g_ref = mlp.loss_and_grad(p, x, y, BOX, ym, ys)
    g, loss = net.grad(1, cuda32(x), cuda32(y))
    g = g.cpu().double().numpy()
    net.check()
    assert abs(float(loss.item()) - loss_ref) <= 2e-3 * loss_ref
    # per weight / bias block: relative Frobenius error <= 1e-2, and element by element
    # |a - r| <= 2^-6 |r| + 2^-8 max |r| -- the oracle rounds at the kernels' points (bf16
    # activations and stage gradients, 2^-9 relative), so elements differ by accumulation
    # order and by the rare bf16 rounding that lands on the other side of a tie (2^-8);
    # one wrong element, e.g. a bias with a flipped sign, exceeds it
    o, worst = 0, 0.0
    for (wo, wi), (bo,) in mlp.param_shapes():
        for n in (wo * wi, bo):
            a, r = g[o:o + n], g_ref[o:o + n]
            assert np.linalg.norm(a - r) <= 1e-2 * np.linalg.norm(r), (o, n)
            bound = 2.0 ** -6 * np.abs(r) + 2.0 ** -8 * np.abs(r).max()
            worst = max(worst, float((np.abs(a - r) / bound).max()))
            assert np.all(np.abs(a - r) <= bound), (o, n, np.abs(a - r).max())
            o += n
    print("B = %d: worst element error / bound %.3g" % (B, worst))


def test_gradient_with_index_gather(net):
    p = params(5)
    net.set_params(0, p)
    net.set_scaling(np.zeros(3), np.ones(3))
    x = workloads.surrogate_inputs(3000, seed=21).astype(np.float32)
    y = np.random.default_rng(1).normal(0, 1, (3000, 3)).astype(np.float32)
    idx = np.random.default_rng(2).permutation(3000)[:1024]
    ga, la = net.grad(0, cuda32(x[idx]), cuda32(y[idx]))
    ga, la = ga.clone(), float(la.item())
    gb, lb = net.grad(0, cuda32(x), cuda32(y), idx=torch.tensor(idx, device="cuda"))
    np.testing.assert_array_equal(ga.cpu().numpy(), gb.cpu().numpy())
    assert abs(la - float(lb.item())) <= 1e-12 * la  # block sums added in any order


def test_adam_matches_oracle(net):
    p = params(6)
    net.set_params(0, p)
    net.set_scaling(np.zeros(3), np.ones(3))
    x = workloads.surrogate_inputs(512, seed=7).astype(np.float32)
    y = np.random.default_rng(3).normal(0, 1, (512, 3)).astype(np.float32)
    cur = p.copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    net.steps[0] = 0
    for t in range(1, 4):
        g, _ = net.grad(0, cuda32(x), cuda32(y))
        gh = g.cpu().double().numpy()
        net.adam(0, 1e-3)
        cur, m, v = mlp.adam_step(cur, gh, m, v, t, 1e-3)
        got = net.get_params(0).cpu().double().numpy()
        np.testing.assert_allclose(got, cur, rtol=1e-5, atol=1e-7)
        cur = got  # continue from the device's FP32 parameters


def test_gate_matches_oracle(net):
    rng = np.random.default_rng(8)
    B = 5000
    x = workloads.surrogate_inputs(B, seed=9, outside_share=0.1).astype(np.float32)
    ym = rng.normal(0, 1, (2, B, 3)).astype(np.float32)
    ym[:, ::3] *= 1e-3  # a third of the samples agree closely
    tau = 0.05
    spread = torch.empty(B, dtype=torch.float32, device="cuda")
    mean, fb, cnt = net.gate(cuda32(x), cuda32(ym), tau, spread=spread)
    mean_ref, fb_ref = mlp.gate(ym.astype(np.float64), x.astype(np.float64), BOX, tau)
    y64 = ym.astype(np.float64)
    std = np.sqrt(((y64 - y64.mean(0)) ** 2).mean(0)).max(axis=1)
    # the kernel's statistic is the population standard deviation in FP32 (two members here)
    np.testing.assert_allclose(spread.cpu().numpy(), std, rtol=1e-5, atol=1e-7)
    far = np.abs(std - tau) > 1e-5
    np.testing.assert_array_equal(fb.cpu().numpy()[far].astype(bool), fb_ref[far])
    assert int(cnt.item()) == int(fb.cpu().numpy().sum())
    np.testing.assert_allclose(mean.cpu().numpy(), mean_ref, rtol=1e-6, atol=1e-7)


def test_training_reduces_loss_and_beats_the_mean_predictor():
    """A short training run on solver data: the standardised MSE of predicting the mean is 1;
    the trained members must get well below it on held-out samples."""
    from paper_2304_06835_gb300 import EnsembleSolver, SurrogateMLP
    N = 32768
    x = workloads.surrogate_inputs(N + 4096, seed=31)
    s = EnsembleSolver("lorenz")
    P = torch.tensor(x[:, :3], device="cuda")
    U = torch.tensor(x[:, 3:], device="cuda")
    T = torch.tensor(np.tile([0.0, 1.0], (len(x), 1)), device="cuda")
    u1, st, _ = s.solve(P, U, T, alg="tsit5", abstol=1e-10, reltol=1e-10)
    assert int(st.abs().sum()) == 0
    y = u1.float()
    xs = torch.tensor(x, dtype=torch.float32, device="cuda")
    net = SurrogateMLP(workloads.surrogate_box(), members=2, batch_max=4096, seed=11)
    yt = y[:N].double().cpu().numpy()
    net.set_scaling(yt.mean(0), yt.std(0))
    hist = net.train(xs[:N], y[:N], epochs=6, batch=1024, lr=2e-3)
    assert hist[-1] < 0.25 and all(b < a for a, b in zip(hist, hist[1:])), hist
    pred = net.forward(xs[N:]).double()
    t = (y[N:].double() - torch.tensor(yt.mean(0), device="cuda")) / \
        torch.tensor(yt.std(0), device="cuda")
    z = (pred - torch.tensor(yt.mean(0), device="cuda")) / torch.tensor(yt.std(0), device="cuda")
    mse = ((z - t[None]) ** 2).mean(dim=(1, 2)).cpu().numpy()
    assert np.all(mse < 0.2), mse
    net.close()
