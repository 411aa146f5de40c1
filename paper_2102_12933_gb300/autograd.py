"""torch.autograd.Function wrappers over the library's hand-written adjoint.

Residual.apply(w, mesh, precision) -> dw/dt at the state w ([nv][4] CUDA
float64 tensor); its backward is fdu_residual_vjp.  RKSteps.apply(w0, mesh,
dt, n_steps, checkpoint_every, precision) -> the state after n_steps SSP-RK3
steps; its backward is fdu_adjoint_rk (checkpointed recomputation).
precision is 64 (FP64) or 48 (the FP64 result with double-word increments):
it selects the forward residual or steps and the adjoint's precision of the
backward pass.  The forward and backward passes both run in the library's
kernels; torch only carries the tensors.
"""
from __future__ import annotations

import torch


def _check_precision(precision):
    if precision not in (64, 48):
        raise ValueError("precision must be 64 or 48")


class _AdjointPrecision:
    """Sets the mesh's adjoint precision for a backward pass and restores it."""

    def __init__(self, mesh, precision):
        self.mesh, self.precision = mesh, precision

    def __enter__(self):
        self.saved = self.mesh.adjoint_precision
        self.mesh.set_adjoint_precision(self.precision)

    def __exit__(self, *exc):
        self.mesh.set_adjoint_precision(self.saved)
        return False


def _check_state(w, mesh):
    if not (w.is_cuda and w.dtype == torch.float64 and tuple(w.shape) == (mesh.nv, 4)):
        raise ValueError("expected a CUDA float64 tensor of shape (nv, 4)")


class Residual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, mesh, precision=64):
        _check_state(w, mesh)
        _check_precision(precision)
        w = w.contiguous()
        mesh.set_state(w)
        out = torch.empty_like(w)
        mesh.residual(precision, out=out)
        ctx.mesh, ctx.precision = mesh, precision
        ctx.save_for_backward(w)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (w,) = ctx.saved_tensors
        mesh = ctx.mesh
        mesh.set_state(w)
        g = torch.empty_like(w)
        with _AdjointPrecision(mesh, ctx.precision):
            mesh.residual_vjp(grad_out.contiguous(), out=g)
        return g, None, None


class RKSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w0, mesh, dt, n_steps, checkpoint_every=10, precision=64):
        _check_state(w0, mesh)
        _check_precision(precision)
        w0 = w0.contiguous()
        mesh.set_state(w0)
        mesh.rk_steps(dt, n_steps, precision)
        out = torch.empty_like(w0)
        mesh.get_state(out=out)
        ctx.mesh, ctx.dt, ctx.n_steps, ctx.k, ctx.precision = mesh, dt, n_steps, checkpoint_every, precision
        ctx.save_for_backward(w0)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (w0,) = ctx.saved_tensors
        mesh = ctx.mesh
        mesh.set_state(w0)
        g = torch.empty_like(w0)
        with _AdjointPrecision(mesh, ctx.precision):
            mesh.adjoint_rk(ctx.dt, ctx.n_steps, grad_out.contiguous(), out=g, checkpoint_every=ctx.k)
        return g, None, None, None, None, None
