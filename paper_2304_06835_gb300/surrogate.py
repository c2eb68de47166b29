"""The learned surrogate (an addition to the paper's ensemble method): an ensemble of BF16
multilayer perceptrons 6 -> 256 -> 256 -> 256 -> 3 that map a Lorenz problem
(sigma, rho, beta, u0) to u(tf), trained on solver output, with a disagreement / out-of-box
gate that sends doubtful samples back to the solver.

Every network operation runs in libens.so's kernels (tcgen05 tensor-core GEMMs and their
fused epilogues, Adam, the gate); this module marshals tensors and drives the training loop.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


class SurrogateMLP:
    """`members` networks sharing one input box.  box: [6, 2] (lo, hi) of
    (sigma, rho, beta, u0_1, u0_2, u0_3)."""

    def __init__(self, box, members=4, batch_max=8192, seed=0, device="cuda"):
        self.device = torch.device(device)
        self.members = int(members)
        self.batch_max = int(batch_max)
        self.box = np.ascontiguousarray(box, dtype=np.float64).reshape(6, 2)
        h = ctypes.c_void_p()
        bx = self.box.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _lib.check(_lib.lib().ens_mlp_create(ctypes.byref(h), self.members, self.batch_max, bx,
                                             int(seed) & 0xFFFFFFFFFFFFFFFF,
                                             _stream(self.device)))
        self._h = h
        self.n_params = int(_lib.lib().ens_mlp_n_params())
        self.steps = [0] * self.members
        self._loss = torch.zeros(1, dtype=torch.float64, device=self.device)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().ens_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scaling(self, y_mean, y_std):
        m = np.ascontiguousarray(y_mean, dtype=np.float64)
        s = np.ascontiguousarray(y_std, dtype=np.float64)
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.check(_lib.lib().ens_mlp_set_scaling(self._h, m.ctypes.data_as(dp),
                                                  s.ctypes.data_as(dp), _stream(self.device)))
        self.y_mean, self.y_std = m, s

    def get_params(self, member):
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().ens_mlp_params(self._h, member, _ptr(out), None,
                                             _stream(self.device)))
        return out

    def set_params(self, member, flat):
        flat = torch.as_tensor(flat, dtype=torch.float32, device=self.device).contiguous()
        if flat.numel() != self.n_params:
            raise ValueError("expected %d parameters" % self.n_params)
        _lib.check(_lib.lib().ens_mlp_params(self._h, member, None, _ptr(flat),
                                             _stream(self.device)))
        torch.cuda.current_stream(self.device).synchronize()

    @staticmethod
    def _xy(x, y=None):
        x = x.contiguous()
        if x.dtype != torch.float32 or x.dim() != 2 or x.shape[1] != 6 or not x.is_cuda:
            raise ValueError("x must be a CUDA float32 tensor [B, 6]")
        if y is not None:
            y = y.contiguous()
            if y.dtype != torch.float32 or tuple(y.shape) != (x.shape[0], 3):
                raise ValueError("y must be a CUDA float32 tensor [B, 3]")
        return x, y

    def grad(self, member, x, y, idx=None, want=True):
        """Gradient of the standardised MSE of one member on a minibatch: rows idx of (x, y)
        (int64 device tensor) or all rows (B <= batch_max).  Returns (grad [n_params] or None,
        loss tensor (device, float64))."""
        x, y = self._xy(x, y)
        B = x.shape[0] if idx is None else idx.numel()
        if idx is not None and (idx.dtype != torch.int64 or not idx.is_cuda):
            raise ValueError("idx must be a CUDA int64 tensor")
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.device) if want else None
        _lib.check(_lib.lib().ens_mlp_grad(self._h, member, B, _ptr(x), _ptr(y),
                                           _ptr(None if idx is None else idx.contiguous()),
                                           _ptr(g), _ptr(self._loss), _stream(self.device)))
        return g, self._loss

    def adam(self, member, lr):
        self.steps[member] += 1
        _lib.check(_lib.lib().ens_mlp_adam(self._h, member, float(lr), self.steps[member],
                                           _stream(self.device)))

    def forward(self, x, member=-1, out=None, layerwise=False):
        """y [E', B, 3] for one member (E' = 1) or all (member = -1): by default the fused
        on-chip kernel, layerwise=True the layer-by-layer path (identical results)."""
        x, _ = self._xy(x)
        E = self.members if member < 0 else 1
        if out is None:
            out = torch.empty((E, x.shape[0], 3), dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().ens_mlp_forward(self._h, member, x.shape[0], _ptr(x), _ptr(out),
                                              1 if layerwise else 0, _stream(self.device)))
        return out

    def gate(self, x, y_members, tau, mean=None, fallback=None, count=None, compact=None,
             t0=0.0, t1=1.0, spread=None):
        """(mean [B, 3], fallback uint8 [B], n_fallback device counter).  compact: optional
        dict of device buffers index int64 [B], params / u0 float32 [B, 3], tspan [B, 2] that
        receive the fallback samples as a row-major solver problem on [t0, t1].  spread:
        optional float32 [B] that receives the members' disagreement the gate compares with
        tau (the largest per-component population standard deviation)."""
        x, _ = self._xy(x)
        B = x.shape[0]
        if mean is None:
            mean = torch.empty((B, 3), dtype=torch.float32, device=self.device)
        if fallback is None:
            fallback = torch.empty(B, dtype=torch.uint8, device=self.device)
        if count is None:
            count = torch.zeros(1, dtype=torch.int64, device=self.device)
        c = compact or {}
        _lib.check(_lib.lib().ens_mlp_gate(
            self._h, B, _ptr(x), _ptr(y_members.contiguous()), float(tau), _ptr(mean),
            _ptr(spread), _ptr(fallback), _ptr(count), _ptr(c.get("index")), _ptr(c.get("params")),
            _ptr(c.get("u0")), _ptr(c.get("tspan")), float(t0), float(t1), _stream(self.device)))
        return mean, fallback, count

    def scatter(self, n, index, u, y):
        """y[index[i]] = u[i] for i < n."""
        _lib.check(_lib.lib().ens_mlp_scatter(int(n), _ptr(index), _ptr(u.contiguous()), _ptr(y),
                                              _stream(self.device)))

    def check(self):
        _lib.check(_lib.lib().ens_mlp_check(self._h, _stream(self.device)))

    def train(self, x, y, *, epochs=10, batch=4096, lr=1e-3, lr_min=1e-5, members=None,
              seed=0, log_every=0):
        """Adam on minibatches of a shuffled (per member) training set with cosine decay of the
        learning rate from lr to lr_min.  Returns the mean minibatch loss of every epoch."""
        x, y = self._xy(x, y)
        N = x.shape[0]
        batch = min(batch, self.batch_max)
        members = range(self.members) if members is None else members
        steps_per_epoch = N // batch
        total = max(1, epochs * steps_per_epoch)
        hist = []
        gen = torch.Generator(device=self.device)
        gen.manual_seed(int(seed))
        for ep in range(epochs):
            ep_loss = torch.zeros(1, dtype=torch.float64, device=self.device)
            for mb in members:
                perm = torch.randperm(N, device=self.device, generator=gen)
                for k in range(steps_per_epoch):
                    idx = perm[k * batch:(k + 1) * batch]
                    step = ep * steps_per_epoch + k
                    cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * step / total))
                    _, loss = self.grad(mb, x, y, idx=idx, want=False)
                    ep_loss += loss
                    self.adam(mb, cur)
            hist.append(float(ep_loss.item()) / (steps_per_epoch * len(list(members))))
            if log_every and (ep + 1) % log_every == 0:
                print("epoch %d loss %.3e" % (ep + 1, hist[-1]))
        self.check()
        return hist


def lorenz_u1(solver, x, *, t1=1.0, tol=1e-10, dtype=torch.float64):
    """u(t1) of the Lorenz problems x [N, 6] = (sigma, rho, beta, u0) by the adaptive Tsit5
    solver (structure-of-arrays inputs), as float32 [N, 3]."""
    xd = x.to(dtype)
    P = xd[:, :3].t().contiguous()
    U = xd[:, 3:].t().contiguous()
    N = x.shape[0]
    T = torch.zeros((2, N), dtype=dtype, device=x.device)
    T[1] = t1
    out, st, _ = solver.solve(P, U, T, alg="tsit5", layout="soa", abstol=tol, reltol=tol)
    return out.t().float().contiguous(), st


def calibrate_tau(net, x_val, y_val, max_err):
    """Largest gate threshold tau for which every validation sample with member spread <= tau
    has a mean-prediction error (max over components) <= max_err.  The spread and the mean
    are the gate kernel's own (ens_mlp_gate), so the threshold is calibrated on the statistic
    the gate compares with it."""
    ym = net.forward(x_val)
    B = ym.shape[1]
    spread_d = torch.empty(B, dtype=torch.float32, device=ym.device)
    mean_d, _, _ = net.gate(x_val, ym, float("inf"), spread=spread_d)
    spread = spread_d.cpu().numpy().astype(np.float64)
    err = np.abs(mean_d.cpu().numpy().astype(np.float64)
                 - y_val.cpu().numpy().astype(np.float64)).max(axis=1)
    order = np.argsort(spread)
    bad = np.flatnonzero(err[order] > max_err)
    if bad.size == 0:
        return float(spread.max()) * 1.0001
    k = bad[0]
    return float(spread[order[k - 1]]) if k > 0 else 0.0


class GatedSurrogate:
    """Surrogate prediction with fallback: the mean of the members where they agree (spread
    <= tau) and the input lies in the training box, the solver (FP32 adaptive Tsit5 at
    fallback_tol) everywhere else."""

    def __init__(self, net, solver, tau, *, t1=1.0, fallback_tol=1e-6):
        self.net, self.solver, self.tau, self.t1 = net, solver, float(tau), t1
        self.fallback_tol = fallback_tol
        self._cap = 0

    def _buffers(self, B):
        if B > self._cap:
            dev = self.net.device
            self._ym = torch.empty((self.net.members, B, 3), dtype=torch.float32, device=dev)
            self._mean = torch.empty((B, 3), dtype=torch.float32, device=dev)
            self._fb = torch.empty(B, dtype=torch.uint8, device=dev)
            self._cnt = torch.zeros(1, dtype=torch.int64, device=dev)
            self._cp = {"index": torch.empty(B, dtype=torch.int64, device=dev),
                        "params": torch.empty((B, 3), dtype=torch.float32, device=dev),
                        "u0": torch.empty((B, 3), dtype=torch.float32, device=dev),
                        "tspan": torch.empty((B, 2), dtype=torch.float32, device=dev)}
            self._cap = B

    def predict(self, x):
        """(y [B, 3] float32, fallback uint8 [B], number of fallbacks).  The outputs are views
        of buffers reused by the next call."""
        B = x.shape[0]
        self._buffers(B)
        ym = self.net.forward(x, out=self._ym[:, :B] if B == self._cap else None)
        self._cnt.zero_()
        mean, fb, cnt = self.net.gate(x, ym, self.tau, mean=self._mean[:B], fallback=self._fb[:B],
                                      count=self._cnt, compact=self._cp, t0=0.0, t1=self.t1)
        n = int(cnt.item())
        if n:
            c = self._cp
            u, _, _ = self.solver.solve(c["params"][:n], c["u0"][:n], c["tspan"][:n], alg="tsit5",
                                        abstol=self.fallback_tol, reltol=self.fallback_tol)
            self.net.scatter(n, c["index"], u, mean)
        return mean, fb, n
