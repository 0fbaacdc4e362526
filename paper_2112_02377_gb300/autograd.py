"""Differentiation through the Jacobi solve (the adjoint method).

``jacobi_solve(rowptr, col, val, b, ...)`` returns x with A x = b solved by the
library's synchronous Jacobi iteration and, under autograd, propagates a loss
gradient g = dL/dx back to the inputs:

    A^T lambda = g            (solved by the same Jacobi iteration on A^T)
    dL/db      = lambda
    dL/dA_ij   = -lambda_i x_j   for every stored entry (i, j) of A

(differentiating A x = b gives A dx = db - dA x).  Both solves and the
gradient kernel run in the CUDA library; this module only marshals tensors.

A forward or adjoint solve that reaches maxit before tol raises
JacobiError(JAC_ENOTCONV): an unconverged x (or lambda) would give a loss
and gradients of a different problem, so neither is returned.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import jacobi as J


class _Handle:
    """Owns a jac_ctx; frees it when dropped (e.g. when backward never runs)."""

    def __init__(self, ctx):
        self.ctx = ctx

    def release(self):
        if self.ctx:
            J.jac_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class JacSolve(torch.autograd.Function):
    """The solve as a torch.autograd.Function:
    ``JacSolve.apply(val, b, rowptr, col, tol, maxit, nparts, x0, opts)``
    (``jacobi_solve`` is the keyword-argument form)."""

    @staticmethod
    def forward(ctx, val, b, rowptr, col, tol, maxit, nparts, x0, extra):
        n = rowptr.numel() - 1
        o = J.opts(**extra)
        fwd = J.jac_setup((rowptr, col, val), b, J.JAC_BANDROW, nparts, o)
        try:
            if x0 is not None:
                J.jac_set_x(fwd, x0)
            k, rel, st = J.jac_solve(fwd, tol, maxit, raise_on_notconv=True)
            x = torch.empty(n, dtype=torch.float64, device=b.device)
            J.jac_get_x(fwd, x)
        except Exception:
            J.jac_free(fwd)
            raise
        ctx.fwd = _Handle(fwd)
        ctx.setup = (tol, maxit, nparts, extra)
        ctx.info = {"sweeps": k, "relres": rel, "status": st}
        ctx.save_for_backward(val, rowptr, col, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        val, rowptr, col, x = ctx.saved_tensors
        tol, maxit, nparts, extra = ctx.setup
        n = rowptr.numel() - 1
        gx = gx.contiguous().to(torch.float64)
        o = J.opts(transpose=1, **extra)
        adj = J.jac_setup((rowptr, col, val), gx, J.JAC_BANDROW, nparts, o)
        try:
            J.jac_solve(adj, tol, maxit, raise_on_notconv=True)
            lam = torch.empty(n, dtype=torch.float64, device=gx.device)
            J.jac_get_x(adj, lam)
        finally:
            J.jac_free(adj)
        dval = None
        if ctx.needs_input_grad[0]:
            dval = torch.empty_like(val)
            J.jac_adjoint_grad(ctx.fwd.ctx, lam, x, dval)
        ctx.fwd.release()
        return dval, lam, None, None, None, None, None, None, None


def jacobi_solve(rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, b: torch.Tensor,
                 tol: float = 1e-12, maxit: int = 1_000_000, nparts: int = 1,
                 x0: Optional[torch.Tensor] = None, **opts) -> torch.Tensor:
    """x = A^{-1} b by synchronous Jacobi, differentiable in ``val`` and ``b``.

    rowptr/col: int32 CUDA tensors (0-based CSR of A, diagonal stored);
    val, b: float64 CUDA tensors.  ``tol`` applies to both the forward solve
    and the adjoint solve (relative 2-norm of the residual); ``x0`` warm-starts
    the forward solve.  Extra keyword arguments are jac_opts fields.
    """
    return JacSolve.apply(val, b, rowptr, col, float(tol), int(maxit), int(nparts), x0, opts)
