"""torch.autograd.Function wrappers over the library's hand-written adjoint.

Residual.apply(w, mesh) -> dw/dt at the state w (FP64, [nv][4] CUDA tensor);
its backward is fdu_residual_vjp.  RKSteps.apply(w0, mesh, dt, n_steps,
checkpoint_every) -> the state after n_steps SSP-RK3 steps; its backward is
fdu_adjoint_rk (checkpointed recomputation).  The forward and backward
passes both run in the library's kernels; torch only carries the tensors.
"""
from __future__ import annotations

import torch


def _check_state(w, mesh):
    if not (w.is_cuda and w.dtype == torch.float64 and tuple(w.shape) == (mesh.nv, 4)):
        raise ValueError("expected a CUDA float64 tensor of shape (nv, 4)")


class Residual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, mesh):
        _check_state(w, mesh)
        w = w.contiguous()
        mesh.set_state(w)
        out = torch.empty_like(w)
        mesh.residual(64, out=out)
        ctx.mesh = mesh
        ctx.save_for_backward(w)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (w,) = ctx.saved_tensors
        mesh = ctx.mesh
        mesh.set_state(w)
        g = torch.empty_like(w)
        mesh.residual_vjp(grad_out.contiguous(), out=g)
        return g, None


class RKSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w0, mesh, dt, n_steps, checkpoint_every=10):
        _check_state(w0, mesh)
        w0 = w0.contiguous()
        mesh.set_state(w0)
        mesh.rk_steps(dt, n_steps, 64)
        out = torch.empty_like(w0)
        mesh.get_state(out=out)
        ctx.mesh, ctx.dt, ctx.n_steps, ctx.k = mesh, dt, n_steps, checkpoint_every
        ctx.save_for_backward(w0)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (w0,) = ctx.saved_tensors
        mesh = ctx.mesh
        mesh.set_state(w0)
        g = torch.empty_like(w0)
        mesh.adjoint_rk(ctx.dt, ctx.n_steps, grad_out.contiguous(), out=g, checkpoint_every=ctx.k)
        return g, None, None, None, None
