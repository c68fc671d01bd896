"""Differentiable solve: u = K^-1 f as a torch.autograd.Function.

K is symmetric, so the adjoint of the solve is the same solve: for a loss J
with dJ/du = w, dJ/df = lambda with K lambda = w (the adjoint A-DEF2 PCG run
on the same context, through the same C ABI).  Gradients with respect to K
itself are not provided here.
"""
import torch


class DeflatedSolve(torch.autograd.Function):
    """u = solver.solve(f, tol); backward: lambda = solver.solve(grad_u, tol)."""

    @staticmethod
    def forward(ctx, f, solver, tol):
        u, info = solver.solve(f.detach().contiguous(), tol=tol)
        ctx.solver = solver
        ctx.tol = tol
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, grad_u):
        lam, _ = ctx.solver.solve(grad_u.detach().contiguous(), tol=ctx.tol)
        return lam, None, None


def solve(solver, f, tol=1e-8):
    """Differentiable u = K^-1 f (f: CUDA float64 tensor, may require grad)."""
    return DeflatedSolve.apply(f, solver, tol)
