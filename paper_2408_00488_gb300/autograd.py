"""torch.autograd wrapper of the solve: gradients of a real loss with respect
to the right-hand side f and the coefficient samples, by one adjoint MINRES
solve (K + conj(lambda) I) Y = G with G = dL/dRe z + i dL/dIm z (the transposed
block system of Eq. 2; A is symmetric) and the per-face formula
dL/da_e = -h^{-2} Re(conj(D_e Y) D_e z), both evaluated in libcsl.so."""
from __future__ import annotations

import torch

from ._binding import Plan


class CSLSolve(torch.autograd.Function):
    """z = CSLSolve.apply(f, lam, tol, maxit, precision, *faces)."""

    @staticmethod
    def forward(ctx, f, lam, tol, maxit, precision, *faces):
        plan = Plan(faces, lam, precision=precision)
        z, info = plan.solve(f.contiguous(), tol=tol, maxit=maxit)
        ctx.plan = plan
        ctx.tol = tol
        ctx.maxit = maxit
        ctx.info = info
        ctx.save_for_backward(z)
        return z

    @staticmethod
    def backward(ctx, grad_z):
        (z,) = ctx.saved_tensors
        plan = ctx.plan
        y, info = plan.adjoint(grad_z.contiguous(), tol=ctx.tol, maxit=ctx.maxit)
        ctx.adjoint_info = info
        gfaces = plan.coef_grad(z, y)
        # the plan lives as long as the autograd graph (backward may run more
        # than once with retain_graph); Plan.__del__ releases it
        return (y, None, None, None, None) + tuple(gfaces)


def solve(f, faces, lam, tol=1e-8, maxit=1000, precision="fp64"):
    """Differentiable solve of (K + lam I) z = f (see CSLSolve)."""
    return CSLSolve.apply(f, lam, tol, maxit, precision, *faces)
