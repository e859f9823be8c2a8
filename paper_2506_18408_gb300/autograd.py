"""Differentiation of x = A^{-1} b through the sketched-FGMRES solver.

The derivative is implicit (not back-propagation through the iterations): for a loss L(x) with g = dL/dx,
lambda = A^{-T} g solves the adjoint system, dL/db = lambda and dL/dA_ij = -lambda_i x_j on the stored entries of A
only.  Both the forward solves and the adjoint solves run in the CUDA library (sfgmres_solve, sfgmres_solve_transpose
with the same sketch and parameters), and the pattern gradient is accumulated by sfgmres_pattern_outer.  Several
right-hand sides (rows of b) are solved together as one batch (sfgmres_solve_batch, nrhs = rows of b): every row is
still its own FGMRES problem with its own stop rules, and gets the result a separate solve would give.
"""
from __future__ import annotations

import torch

from .sfgmres import BREAKDOWN, NOT_CONVERGED


def _solve_rows(solver, B, X, m, s, k, tol, transpose):
    """X[r] = A^{-1} B[r] (A^{-T} with ``transpose``) for every row, as one batch; raises if a row fails."""
    what = "adjoint" if transpose else "forward"
    if B.shape[0] == 1:
        _, info = solver.solve(B[0], m=m, s=s, k=k, tol=tol, out=X[0], transpose=transpose)
        if info["status"] in (NOT_CONVERGED, BREAKDOWN):
            raise RuntimeError(f"sfgmres {what} solve did not converge: {info['rel_res_true']:.3e}")
        return
    _, info = solver.solve_batch(B.reshape(-1), nrhs=B.shape[0], m=m, s=s, k=k, tol=tol, out=X.reshape(-1),
                                 transpose=transpose)
    for r, st in enumerate(info["status_p"]):
        if st in (NOT_CONVERGED, BREAKDOWN):
            raise RuntimeError(f"sfgmres {what} solve {r} did not converge: {info['rel_res_true_p'][r]:.3e}")


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
        _solve_rows(solver, B, X, m, s, k, tol, transpose=False)
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
        _solve_rows(solver, G, Lam, m, s, k, tol, transpose=True)
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
