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


class ComplianceSteps(torch.autograd.Function):
    """J = sum_s f_s^T u_s over successive crack-front systems K_s u_s = f_s
    (one solver per step; the steps share the elements' moduli), with no u
    kept between forward and backward: the backward solves every step again
    (u recomputed, not stored).  For the compliance the adjoint solution is u
    itself, so that one solve per step gives dJ/df_s = 2 u_s and
    dJ/dE_e = sum_s -u_s,e^T Khat_s,e u_s,e (each step's own element data)."""

    @staticmethod
    def forward(ctx, young, tol, solvers, elements, *fs):
        J = None
        for s, f in zip(solvers, fs):
            u, _ = s.solve(f.detach().contiguous(), tol=tol)
            Js = torch.dot(f.detach(), u)
            J = Js if J is None else J + Js
            del u
        ctx.solvers, ctx.elements, ctx.tol = solvers, elements, tol
        ctx.save_for_backward(*fs)          # the inputs only
        return J

    @staticmethod
    def backward(ctx, gJ):
        fs = ctx.saved_tensors
        grad_young = None
        grads_f = []
        for i, (s, f) in enumerate(zip(ctx.solvers, fs)):
            u, _ = s.solve(f.detach().contiguous(), tol=ctx.tol)     # recomputed
            if ctx.needs_input_grad[0]:
                g = s.element_sensitivity(ctx.elements[i], u, u)
                grad_young = g if grad_young is None else grad_young + g
            grads_f.append(2.0 * gJ * u if ctx.needs_input_grad[4 + i] else None)
            del u
        if grad_young is not None:
            grad_young = gJ * grad_young
        return (grad_young, None, None, None, *grads_f)


def compliance_steps(solvers, loads, tol=1e-8, young=None, elements=None):
    """Total compliance sum_s f_s^T K_s^-1 f_s of successive crack-front
    systems, differentiable in the loads and (with young and one Elements per
    step) in the element moduli, recomputing each u_s in the backward instead
    of storing it."""
    if len(solvers) != len(loads):
        raise ValueError("one load per solver")
    if young is not None and (elements is None or len(elements) != len(solvers)):
        raise ValueError("young needs one Elements per step")
    return ComplianceSteps.apply(young, tol, list(solvers), elements, *loads)
