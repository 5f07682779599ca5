"""torch.autograd.Functions over the library's sweeps and their adjoints.

ConstStencilFn.apply(u0, plan, adjoint_plan, T) returns u^T for a
constant-weight plan; its backward sweeps the transposed stencil (the
reflected weights w_{-o}, same boundary rule: the transpose of the zero-ghost
and of the periodic operator) T steps over the upstream gradient.
`sweep(u0, dims, radius, weights, boundary, T)` builds both plans.

StencilAdjointFn.apply(u0, kappa, plan, dt, T, ckpt_every) returns u^T, the
field after T explicit steps of du/dt = div(kappa grad u) (the paper's Eq. 1
with a per-cell diffusivity).  Its backward takes the upstream gradient
dL/du^T as lambda^T and sweeps the transposed stencil backward in time
(stencil_adjoint_vjp), recomputing the forward states from checkpoints every
ckpt_every steps (0: every state kept when it fits in half of the free
device memory, else about sqrt(T)).  dt is a constant (no gradient).  Every
step runs in the library's CUDA kernels.
"""
import numpy as np
import torch

from . import Plan, stencil_adjoint_vjp, stencil_run


class StencilAdjointFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, kappa, plan, dt, T, ckpt_every=0):
        u = u0.detach().clone().contiguous()
        stencil_run(plan.handle, u, T, kappa.detach().contiguous(), dt)
        ctx.save_for_backward(u0.detach(), kappa.detach())
        ctx.plan, ctx.dt, ctx.T, ctx.ckpt = plan, float(dt), int(T), int(ckpt_every)
        return u

    @staticmethod
    def backward(ctx, grad_out):
        u0, kappa = ctx.saved_tensors
        lam = grad_out.detach().contiguous()
        gu = torch.empty_like(u0)
        gk = torch.empty_like(u0)
        stencil_adjoint_vjp(ctx.plan.handle, u0.contiguous(), kappa.contiguous(), ctx.dt, ctx.T,
                            ctx.ckpt, lam, gu, gk)
        return gu, gk, None, None, None, None


def diffuse(u0, kappa, plan, dt, T, ckpt_every=0):
    """u^T with autograd support for u0 and kappa."""
    return StencilAdjointFn.apply(u0, kappa, plan, dt, T, ckpt_every)


def reflected(weights):
    """w_{-o}: the weights of the transposed stencil (every axis reversed)."""
    w = np.asarray(weights, dtype=np.float64)
    return np.ascontiguousarray(w[(slice(None, None, -1),) * w.ndim])


class ConstStencilFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, plan, adjoint_plan, T):
        u = u0.detach().clone().contiguous()
        stencil_run(plan.handle, u, T)
        ctx.adjoint_plan, ctx.T = adjoint_plan, int(T)
        return u

    @staticmethod
    def backward(ctx, grad_out):
        lam = grad_out.detach().clone().contiguous()
        stencil_run(ctx.adjoint_plan.handle, lam, ctx.T)
        return lam, None, None, None


def sweep(u0, dims, radius, weights, boundary, T, plans=None):
    """u^T of a constant-weight stencil with autograd support for u0.  Pass
    `plans` = (plan, adjoint_plan) to reuse plans across calls; otherwise they
    are built here (the adjoint plan takes the reflected weights)."""
    if plans is None:
        plans = (Plan(dims, radius, weights, boundary), Plan(dims, radius, reflected(weights), boundary))
    return ConstStencilFn.apply(u0, plans[0], plans[1], T)
