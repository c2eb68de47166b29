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

    def forward(self, x, member=-1, out=None):
        """y [E', B, 3] for one member (E' = 1) or all (member = -1)."""
        x, _ = self._xy(x)
        E = self.members if member < 0 else 1
        if out is None:
            out = torch.empty((E, x.shape[0], 3), dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().ens_mlp_forward(self._h, member, x.shape[0], _ptr(x), _ptr(out),
                                              _stream(self.device)))
        return out

    def gate(self, x, y_members, tau, mean=None, fallback=None, count=None):
        """(mean [B, 3], fallback uint8 [B], n_fallback device counter)."""
        x, _ = self._xy(x)
        B = x.shape[0]
        if mean is None:
            mean = torch.empty((B, 3), dtype=torch.float32, device=self.device)
        if fallback is None:
            fallback = torch.empty(B, dtype=torch.uint8, device=self.device)
        if count is None:
            count = torch.zeros(1, dtype=torch.int64, device=self.device)
        _lib.check(_lib.lib().ens_mlp_gate(self._h, B, _ptr(x), _ptr(y_members.contiguous()),
                                           float(tau), _ptr(mean), _ptr(fallback), _ptr(count),
                                           _stream(self.device)))
        return mean, fallback, count

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
