"""Reverse-mode differentiation of fixed-step ensemble solves through torch.autograd.

    u_tf = solve_fixed(solver, params, u0, tspan, alg="tsit5_fixed", dt=1e-3)
    loss = ((u_tf - target) ** 2).sum(); loss.backward()   # params.grad, u0.grad

The forward runs ens_adjoint_forward (fixed-step solve + checkpoints every K steps); the
backward runs ens_adjoint, the hand-written discrete adjoint of the Runge-Kutta step map
(the paper's solvers are differentiable, Sec. 6.5).  Gradients are exact for the discrete
map up to rounding.  Only argument marshalling happens here.
"""
from __future__ import annotations

import torch


class _FixedStepSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, u0, tspan, solver, alg, dt, layout, max_steps, every):
        out, ckpt, status, max_steps = solver.adjoint_forward(
            params.detach(), u0.detach(), tspan, alg, dt=dt, layout=layout, max_steps=max_steps,
            checkpoint_every=every)
        ctx.save_for_backward(params, u0, tspan, ckpt)
        ctx.cfg = (solver, alg, dt, layout, max_steps, every)
        ctx.mark_non_differentiable(status)
        return out, status

    @staticmethod
    def backward(ctx, grad_out, _grad_status):
        params, u0, tspan, ckpt = ctx.saved_tensors
        solver, alg, dt, layout, max_steps, every = ctx.cfg
        if grad_out is None:
            return (None,) * 9
        gp, gu = solver.adjoint(params.detach(), u0.detach(), tspan,
                                grad_out.to(params.dtype).contiguous(), alg, dt=dt,
                                layout=layout, max_steps=max_steps, checkpoint_every=every,
                                ckpt=ckpt)
        return gp, gu, None, None, None, None, None, None, None


def solve_fixed(solver, params, u0, tspan, alg="tsit5_fixed", *, dt, layout="rowmajor",
                max_steps=None, checkpoint_every=64, return_status=False):
    """u(tf) of a fixed-step solve (TSIT5_FIXED or RK4), differentiable w.r.t. params and u0."""
    if max_steps is None:
        max_steps = solver.max_steps_of(tspan, dt, layout)
    out, status = _FixedStepSolve.apply(params, u0, tspan, solver, alg, dt, layout,
                                        int(max_steps), int(checkpoint_every))
    return (out, status) if return_status else out
