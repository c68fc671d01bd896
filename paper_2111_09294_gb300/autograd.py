"""Differentiable solve: u = K^-1 f as a torch.autograd.Function.

K is symmetric, so the adjoint of the solve is the same solve: for a loss J
with dJ/du = w, dJ/df = lambda with K lambda = w (the adjoint A-DEF2 PCG run
on the same context, through the same C ABI).  With per-element data, the
gradient with respect to the elements' Young's moduli follows from the same
lambda: K = sum_e E_e Khat_e gives dJ/dE_e = -lambda_e^T Khat_e u_e (one
warp per element in the library).  The moduli are an input of the graph
only: the solver's K must be the one assembled with them.
"""
import torch


class DeflatedSolve(torch.autograd.Function):
    """u = solver.solve(f, tol); backward: lambda = solver.solve(grad_u, tol),
    grad_f = lambda, grad_young = the elements' -lambda_e^T Khat_e u_e."""

    @staticmethod
    def forward(ctx, f, young, solver, tol, elements):
        u, info = solver.solve(f.detach().contiguous(), tol=tol)
        ctx.solver = solver
        ctx.tol = tol
        ctx.elements = elements
        ctx.info = info
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        lam, _ = ctx.solver.solve(grad_u.detach().contiguous(), tol=ctx.tol)
        grad_young = None
        if ctx.needs_input_grad[1]:
            grad_young = ctx.solver.element_sensitivity(ctx.elements, u, lam)
        return lam, grad_young, None, None, None


def solve(solver, f, tol=1e-8, young=None, elements=None):
    """Differentiable u = K^-1 f (f: CUDA float64 tensor, may require grad).
    young (optional, one float64 entry per element, may require grad) with
    elements (an Elements on the same device) adds dJ/dE to the backward."""
    if young is not None and elements is None:
        raise ValueError("young needs the elements' data")
    return DeflatedSolve.apply(f, young, solver, tol, elements)
