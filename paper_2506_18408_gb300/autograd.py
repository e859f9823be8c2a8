"""Differentiation of x = A^{-1} b through the sketched-FGMRES solver.

The derivative is implicit (not back-propagation through the iterations): for a loss L(x) with g = dL/dx,
lambda = A^{-T} g solves the adjoint system, dL/db = lambda and dL/dA_ij = -lambda_i x_j on the stored entries of A
only.  Both the forward solves and the adjoint solves run in the CUDA library (sfgmres_solve, sfgmres_solve_transpose
with the same sketch and parameters), and the pattern gradient is accumulated by sfgmres_pattern_outer.  Several
right-hand sides (rows of b) are solved one after another with the same handle.
"""
from __future__ import annotations

import torch

from .sfgmres import BREAKDOWN, NOT_CONVERGED


class SFGMRESSolve(torch.autograd.Function):
    """``x = SFGMRESSolve.apply(solver, vals, b, m, s, k, tol)``.

    ``solver``: a :class:`Solver` for the sparsity pattern; ``vals``: float64 CUDA tensor ``(nnz,)`` of A's values in
    the solver's stored order; ``b``: float64 CUDA tensor ``(n,)`` or ``(nrhs, n)``.  Returns ``x`` of b's shape.
    Raises if a solve does not reach ``tol`` (the implicit gradient assumes the solution).
    """

    @staticmethod
    def forward(ctx, solver, vals, b, m, s, k, tol):
        solver.update_values(vals.detach().contiguous())
        B = b.detach().reshape(-1, solver.n).contiguous()
        X = torch.empty_like(B)
        for r in range(B.shape[0]):
            _, info = solver.solve(B[r], m=m, s=s, k=k, tol=tol, out=X[r])
            if info["status"] in (NOT_CONVERGED, BREAKDOWN):
                raise RuntimeError(f"sfgmres forward solve {r} did not converge: {info['rel_res_true']:.3e}")
        ctx.solver = solver
        ctx.params = (m, s, k, tol)
        ctx.bshape = b.shape
        ctx.save_for_backward(vals, X)
        return X.reshape(b.shape)

    @staticmethod
    def backward(ctx, gx):
        vals, X = ctx.saved_tensors
        solver = ctx.solver
        m, s, k, tol = ctx.params
        solver.update_values(vals.detach().contiguous())
        G = gx.reshape(-1, solver.n).contiguous().to(torch.float64)
        Lam = torch.empty_like(G)
        for r in range(G.shape[0]):
            if not torch.any(G[r] != 0):
                Lam[r].zero_()
                continue
            _, info = solver.solve(G[r], m=m, s=s, k=k, tol=tol, out=Lam[r], transpose=True)
            if info["status"] in (NOT_CONVERGED, BREAKDOWN):
                raise RuntimeError(f"sfgmres adjoint solve {r} did not converge: {info['rel_res_true']:.3e}")
        gvals = None
        if ctx.needs_input_grad[1]:
            gvals = torch.zeros_like(vals)
            for r in range(G.shape[0]):
                solver.pattern_outer(Lam[r], X[r], -1.0, gvals)
        gb = Lam.reshape(ctx.bshape) if ctx.needs_input_grad[2] else None
        return None, gvals, gb, None, None, None, None


def sfgmres_solve_autograd(solver, vals, b, *, m: int, s: int, k: int, tol: float = 1e-8):
    """Differentiable ``x = A^{-1} b`` (see :class:`SFGMRESSolve`)."""
    return SFGMRESSolve.apply(solver, vals, b, m, s, k, tol)
