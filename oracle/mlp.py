"""NumPy oracle of the learned surrogate -- TEST INFRASTRUCTURE ONLY.

The surrogate is not in the paper (it is an addition to the ensemble method): a small
multilayer perceptron maps a Lorenz problem (sigma, rho, beta, u0) to the state u(tf), with
several independently initialised members whose disagreement gates a fallback to the solver.

What it computes, in the order the kernels compute it (FP64 arithmetic, with the bf16
rounding points the kernels have, so that the two can be compared element by element):

  x_n  = bf16( 2 (x - lo) / (hi - lo) - 1 ), zero-padded to the first layer's padded width
  Z_l  = H_{l-1} bf16(W_l)^T + b_l          (H_0 = x_n; accumulation exact here, FP32 there)
  H_l  = bf16( gelu(Z_l) ),  gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2   (Hendrycks &
         Gimpel 2016, exact erf form)
  yhat = Z_L  (standardised output);  y = yhat * y_std + y_mean

Loss (mean squared error on standardised targets t = (y - y_mean) / y_std):
  L = sum_{b,j} (yhat_bj - t_bj)^2 / (B * n_out)
Backward (reverse of the above):
  dZ_L = bf16( 2 (yhat - t) / (B * n_out) )
  dW_l = dZ_l^T H_{l-1},  db_l = sum_b dZ_l,  dH_{l-1} = dZ_l bf16(W_l)
  dZ_{l-1} = bf16( dH_{l-1} * gelu'(Z_{l-1}) ),  gelu'(z) = Phi(z) + z phi(z)
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
Gate: mean and population standard deviation over the members; fall back to the solver when
any input lies outside the training box or max_j std_j > tau.

``exact=True`` switches every bf16 rounding off (used by the pins against finite differences
and an independent autograd implementation).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

WIDTHS = (6, 256, 256, 256, 3)


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = x.view(np.uint32).astype(np.uint64)
    nan = np.isnan(x)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def _q(a, exact):
    return np.asarray(a, dtype=np.float64) if exact else bf16_round(a)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def pad_width(n):
    return max(16, (n + 15) // 16 * 16)


def param_shapes(widths=WIDTHS):
    """(W_l [out, in], b_l [out]) for l = 1..L; the flat parameter vector concatenates
    W_1, b_1, W_2, b_2, ... in that order, row-major."""
    return [((widths[i + 1], widths[i]), (widths[i + 1],)) for i in range(len(widths) - 1)]


def n_params(widths=WIDTHS):
    return sum(a[0] * a[1] + b[0] for a, b in param_shapes(widths))


def unflatten(flat, widths=WIDTHS):
    flat = np.asarray(flat, dtype=np.float64)
    out, o = [], 0
    for (wo, wi), (bo,) in param_shapes(widths):
        W = flat[o:o + wo * wi].reshape(wo, wi)
        o += wo * wi
        b = flat[o:o + bo]
        o += bo
        out.append((W, b))
    assert o == flat.size
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def normalise(x, box, exact=False):
    lo, hi = box[:, 0], box[:, 1]
    xn = 2.0 * (np.asarray(x, np.float64) - lo) / (hi - lo) - 1.0
    return _q(xn.astype(np.float32) if not exact else xn, exact)


def forward(flat, x, box, y_mean, y_std, widths=WIDTHS, exact=False, keep=False):
    """Surrogate output y [B, n_out] (de-standardised).  keep=True also returns the
    intermediate (H_l, Z_l) lists for the backward pass."""
    layers = unflatten(flat, widths)
    H = [normalise(x, box, exact)]
    Z = []
    for l, (W, b) in enumerate(layers):
        z = H[-1] @ _q(W, exact).T + np.asarray(b, np.float64)
        Z.append(z)
        if l < len(layers) - 1:
            H.append(_q(gelu(z), exact))
    yhat = Z[-1]
    y = yhat * y_std + y_mean
    return (y, H, Z) if keep else y


def loss_and_grad(flat, x, y, box, y_mean, y_std, widths=WIDTHS, exact=False):
    """MSE loss on standardised targets and its gradient (flat, same layout as the params)."""
    layers = unflatten(flat, widths)
    _, H, Z = forward(flat, x, box, y_mean, y_std, widths, exact, keep=True)
    B, n_out = Z[-1].shape
    t = (np.asarray(y, np.float64) - y_mean) / y_std
    r = Z[-1] - t
    loss = float((r * r).sum() / (B * n_out))
    dZ = _q(2.0 * r / (B * n_out), exact)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = (dZ.T @ H[l], dZ.sum(axis=0))
        if l > 0:
            dH = dZ @ _q(W, exact)
            dZ = _q(dH * gelu_grad(Z[l - 1]), exact)
    return loss, flatten(grads)


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def gate(y_members, x, box, tau):
    """y_members [E, B, n_out] -> (mean [B, n_out], fallback bool [B])."""
    ym = np.asarray(y_members, np.float64)
    mean = ym.mean(axis=0)
    std = np.sqrt(((ym - mean) ** 2).mean(axis=0))
    lo, hi = box[:, 0], box[:, 1]
    outside = np.any((x < lo) | (x > hi), axis=1)
    return mean, outside | (std.max(axis=1) > tau)
