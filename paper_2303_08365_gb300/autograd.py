"""torch.autograd.Function over the variable-coefficient sweep and its adjoint.

StencilAdjointFn.apply(u0, kappa, plan, dt, T, ckpt_every) returns u^T, the
field after T explicit steps of du/dt = div(kappa grad u) (the paper's Eq. 1
with a per-cell diffusivity).  Its backward takes the upstream gradient
dL/du^T as lambda^T and sweeps the transposed stencil backward in time
(stencil_adjoint_vjp), recomputing the forward states from checkpoints every
ckpt_every steps (0: every state kept when it fits in half of the free
device memory, else about sqrt(T)).  dt is a constant (no gradient).  Every
step runs in the library's CUDA kernels.
"""
import torch

from . import stencil_adjoint_vjp, stencil_run


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
