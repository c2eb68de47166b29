"""Pins of the surrogate network's oracle (oracle/mlp.py) against independent references:
torch's bf16 conversion, the normal CDF of scipy.stats, torch autograd (an independent
implementation of the same network), central differences, torch.optim.Adam, and closed
forms (gelu(x) - gelu(-x) = x, Adam's first step, the gate's definition on built cases)."""
import math

import numpy as np
import pytest
import torch
from scipy.stats import norm

from oracle import mlp


def test_bf16_round_ties_to_even_and_matches_torch():
    one = 1.0
    assert mlp.bf16_round([one + 2.0 ** -8])[0] == 1.0                  # tie -> even (down)
    assert mlp.bf16_round([one + 3 * 2.0 ** -8])[0] == 1.0 + 2.0 ** -6  # tie -> even (up)
    assert mlp.bf16_round([one + 2.0 ** -8 + 2.0 ** -20])[0] == 1.0 + 2.0 ** -7
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 10, 100000), rng.normal(0, 1e-3, 1000),
                        [0.0, -0.0, 65504.0, 1e-40, -3.3e38]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)


def test_gelu_is_x_times_normal_cdf():
    z = np.linspace(-8, 8, 2001)
    np.testing.assert_allclose(mlp.gelu(z), z * norm.cdf(z), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(mlp.gelu(z) - mlp.gelu(-z), z, rtol=1e-13, atol=1e-14)
    assert abs(mlp.gelu(1.0) - 0.8413447460685429) < 1e-15
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-8, atol=1e-9)


def _random_params(widths, seed):
    rng = np.random.default_rng(seed)
    layers = []
    for (wo, wi), (bo,) in mlp.param_shapes(widths):
        layers.append((rng.normal(0, 1 / math.sqrt(wi), (wo, wi)), rng.normal(0, 0.1, bo)))
    return mlp.flatten(layers)


def _torch_reference(flat, x, y, box, y_mean, y_std, widths):
    layers = mlp.unflatten(flat, widths)
    ps = []
    for W, b in layers:
        ps += [torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)]
    lo, hi = torch.tensor(box[:, 0]), torch.tensor(box[:, 1])
    h = 2 * (torch.tensor(x) - lo) / (hi - lo) - 1
    for i in range(len(layers)):
        h = torch.nn.functional.linear(h, ps[2 * i], ps[2 * i + 1])
        if i < len(layers) - 1:
            h = torch.nn.functional.gelu(h)  # exact erf form
    out = h * torch.tensor(y_std) + torch.tensor(y_mean)
    t = (torch.tensor(y) - torch.tensor(y_mean)) / torch.tensor(y_std)
    loss = ((h - t) ** 2).mean()
    loss.backward()
    g = np.concatenate([p.grad.numpy().ravel() for p in ps])
    return out.detach().numpy(), float(loss.detach()), g


@pytest.mark.parametrize("widths", [(6, 8, 8, 8, 3), mlp.WIDTHS])
def test_exact_forward_and_gradient_match_torch_autograd(widths):
    flat = _random_params(widths, 1)
    rng = np.random.default_rng(2)
    box = np.array([[8, 12], [0, 28], [2, 3], [-5, 5], [-5, 5], [-5, 5]], float)
    x = rng.uniform(box[:, 0], box[:, 1], (64, 6))
    y = rng.normal(0, 3, (64, 3))
    y_mean, y_std = np.array([0.5, -1.0, 2.0]), np.array([2.0, 3.0, 4.0])
    out_t, loss_t, g_t = _torch_reference(flat, x, y, box, y_mean, y_std, widths)
    out = mlp.forward(flat, x, box, y_mean, y_std, widths, exact=True)
    loss, g = mlp.loss_and_grad(flat, x, y, box, y_mean, y_std, widths, exact=True)
    np.testing.assert_allclose(out, out_t, rtol=1e-12, atol=1e-12)
    assert abs(loss - loss_t) <= 1e-12 * max(1, loss_t)
    np.testing.assert_allclose(g, g_t, rtol=1e-10, atol=1e-12)


def test_exact_gradient_matches_central_differences():
    widths = (6, 8, 8, 8, 3)
    flat = _random_params(widths, 3)
    rng = np.random.default_rng(4)
    box = np.array([[0, 1]] * 6, float)
    x = rng.uniform(0, 1, (16, 6))
    y = rng.normal(0, 1, (16, 3))
    ym, ys = np.zeros(3), np.ones(3)
    _, g = mlp.loss_and_grad(flat, x, y, box, ym, ys, widths, exact=True)
    h = 1e-6
    idx = rng.choice(flat.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        lp, _ = mlp.loss_and_grad(flat + e, x, y, box, ym, ys, widths, exact=True)
        lm, _ = mlp.loss_and_grad(flat - e, x, y, box, ym, ys, widths, exact=True)
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-7 * max(1, abs(g[i]))


def test_rounded_forward_close_to_exact():
    """The bf16 rounding points perturb the result by O(2^-8) relative, not more."""
    flat = _random_params(mlp.WIDTHS, 5)
    rng = np.random.default_rng(6)
    box = np.array([[8, 12], [0, 28], [2, 3], [-5, 5], [-5, 5], [-5, 5]], float)
    x = rng.uniform(box[:, 0], box[:, 1], (256, 6))
    a = mlp.forward(flat, x, box, np.zeros(3), np.ones(3))
    b = mlp.forward(flat, x, box, np.zeros(3), np.ones(3), exact=True)
    rel = np.abs(a - b).max() / np.abs(b).max()
    assert 1e-5 < rel < 3e-2


def test_adam_first_step_and_torch():
    rng = np.random.default_rng(7)
    p = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    p1, m, v = mlp.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    # first step: m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    np.testing.assert_allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-15, atol=1e-15)
    pt = torch.tensor(p, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    cur, mm, vv = p.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        gg = rng.normal(0, 1, 50)
        pt.grad = torch.tensor(gg)
        opt.step()
        cur, mm, vv = mlp.adam_step(cur, gg, mm, vv, t, lr=1e-3)
    np.testing.assert_allclose(cur, pt.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_gate_cases():
    box = np.array([[0, 1]] * 6, float)
    x = np.full((4, 6), 0.5)
    x[2, 3] = 1.5                                           # outside the box
    ym = np.zeros((4, 4, 3))
    ym[:, 1, 0] = [1.0, -1.0, 1.0, -1.0]                    # std 1 on component 0
    ym[:, 3, 2] = [0.1, 0.1, 0.1, 0.1]                      # agreement, nonzero mean
    mean, fb = mlp.gate(ym, x, box, tau=0.5)
    assert list(fb) == [False, True, True, False]
    np.testing.assert_allclose(mean[3], [0, 0, 0.1])
    _, fb = mlp.gate(ym, x, box, tau=1.5)
    assert list(fb) == [False, False, True, False]
