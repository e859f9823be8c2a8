"""FGMRES / FFOM with a sketched-GMRES preconditioner, and restarting with a variable preconditioner (oracle side).

TEST INFRASTRUCTURE ONLY.

* :func:`fgmres` follows Algorithm 1 (Section 2) with the preconditioner ``z_j = M_j^{-1} v_j`` given by one
  sGMRES cycle with zero initial guess (Section 3, :func:`oracle.sgmres.sgmres_cycle`).  The outer basis is
  orthogonalised by modified Gram-Schmidt exactly as printed in Algorithm 1 (classical Gram-Schmidt with one
  reorthogonalisation pass as an option).  The FGMRES coefficients are the least-squares solution
  ``y_j = argmin || beta e_1 - H_j y ||`` over the ``(j+1) x j`` Hessenberg matrix (Algorithm 1); FFOM uses
  ``y_j = H_j^{-1} beta e_1``.  The FFOM residual norm is evaluated from Eq. 4, ``h_{j+1,j} |gamma_j|`` with
  ``gamma_j = e_j^T H_j^{-1} beta e_1``, and feeds stop rule C3 of the next inner cycle (Eq. 5 bound,
  ``||r_1|| <= beta ||rhat_1||`` at the first step).
* :func:`restarted` is Algorithm 2: ``z_j = M_j^{-1} r_{j-1}``, ``x_j = x_{j-1} + z_j``.

Stopping (the paper fixes only a relative residual target): the outer loop stops once the least-squares residual
estimate ``|| beta e_1 - H_j y_j ||`` is at most ``tol * ||b||`` and the recomputed true residual
``||b - A x_j||`` confirms it; if the true residual does not confirm it the loop continues while the outer budget
lasts.  ``h_{j+1,j} = 0`` means the iterate is exact (happy breakdown).  The outer loop is never restarted.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional, Sequence

import numpy as np
from scipy.sparse.linalg import LinearOperator

from .sgmres import CycleResult, sgmres_cycle
from .sketch import sketch_matrix
from .lowprec import INNER_DTYPES

CONVERGED = 0
NOT_CONVERGED = 1
BREAKDOWN = 2  # inner cycle produced no correction


@dataclasses.dataclass
class FGMRESResult:
    x: np.ndarray
    status: int
    outer_iters: int
    rel_res_true: float
    est_hist: List[float]  # ||beta e1 - H_j y_j|| / ||b|| per outer step
    ffom_hist: List[float]  # FFOM residual (Eq. 4) / ||b|| per outer step
    inner_k: List[int]
    inner_reason: List[int]
    true_hist: Optional[List[float]] = None  # ||b - A x_j|| / ||b|| per step (if requested)
    V: Optional[np.ndarray] = None
    Z: Optional[np.ndarray] = None
    H: Optional[np.ndarray] = None
    beta: float = 0.0
    cycles: Optional[List[CycleResult]] = None
    rhat_hist: Optional[List[float]] = None  # ||v_j - A z_j|| per step (if requested)
    rho_hist: Optional[List[float]] = None  # sketched residual rho_k each cycle ended with (if requested)


def _sketch_for(n, s, zeta, seed, kind):
    return sketch_matrix(n, s, zeta, seed, kind)


def fgmres(A, b: np.ndarray, x0: Optional[np.ndarray] = None, *, m: int, s: int, t: int, tol: float = 1e-8,
           max_outer: int = 50, sketch_seed: int = 1, zeta: int = 8, sketch_kind: str = "sparse_sign",
           cond_thr: float = 1e15, c3: bool = True, outer_orth: str = "mgs", variant: str = "fgmres",
           inner: str = "fp64", precond: Optional[Callable[[np.ndarray], np.ndarray]] = None,
           record: bool = False, track_true: bool = False,
           right_precond: Optional[Callable[[np.ndarray], np.ndarray]] = None, trace: bool = False,
           level_steps: Sequence[int] = (), _child: bool = False) -> FGMRESResult:
    """Solve ``A x = b`` by FGMRES (or FFOM) preconditioned with sGMRES cycles (Algorithm 1 + Section 3).

    ``A``: scipy sparse (FP64).  ``m``: inner basis size (C1, the paper's ``k_max``); ``t``: Arnoldi truncation;
    ``s``: sketch rows.  ``precond`` replaces the sGMRES cycle by an arbitrary ``v -> z`` (used by the pins).
    ``right_precond`` (``u -> M^{-1} u``, e.g. ILU(0) from :mod:`oracle.ilu`) right-preconditions the inner solver:
    each sGMRES cycle approximates ``(A M^{-1})^{-1} v_j`` and ``z_j`` is ``M^{-1}`` of its result, so the outer
    FGMRES still minimises the residual of ``A x = b`` (FP64 inner cycles only).
    ``trace`` records, per outer step, the true inner residual ``||v_j - A z_j||`` and the sketched residual the
    cycle ended with (the two sides of the Eq. 5 bound and its estimate) without keeping the bases that ``record``
    keeps.

    ``level_steps`` = (J_1, J_2, ...) makes this the top of a multi-level FGMRES (Section 5): the preconditioner of
    step j is an FGMRES run of at most J_1 outer steps on ``A z = v_j`` (zero initial guess), whose own preconditioner
    is an FGMRES run of at most J_2 steps, and so on; the lowest level uses the sGMRES cycle.  A lower level stops
    early once the bound of Eq. 5 predicts that its parent meets the parent's target: with rule C3 on, the child of
    step j solves to the relative tolerance tol ||b|| / ||r~_{j-1}|| (||r~_{-1}|| = beta), the same test C3 applies to
    an sGMRES cycle; with C3 off it runs its full budget.  A lower level always takes at least one step, stops on its
    Givens estimate and returns its last iterate.  For the parent, ``inner_k`` then counts the child's outer steps
    and ``inner_reason`` is 3 (the child met its tolerance) or 1 (budget).
    """
    n = b.shape[0]
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    x0 = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64)
    if nb == 0.0:
        return FGMRESResult(np.zeros(n), CONVERGED, 0, 0.0, [], [], [], [])
    r0 = b - A @ x0
    beta = float(np.linalg.norm(r0))
    if beta <= tol * nb and not _child:
        return FGMRESResult(x0.copy(), CONVERGED, 0, beta / nb, [], [], [], [], beta=beta)

    S = None
    A_in = S_in = None
    if precond is None:
        S = _sketch_for(n, s, zeta, sketch_seed, sketch_kind)
        dt = INNER_DTYPES[inner]
        A_in = A if dt == np.float64 else A.astype(dt)
        S_in = S if dt == np.float64 else S.astype(dt)
        if right_precond is not None:
            if dt != np.float64:
                raise ValueError("right preconditioning needs FP64 inner cycles")
            A_in = LinearOperator((n, n), matvec=lambda u: A @ right_precond(u), dtype=np.float64)

    V = np.zeros((n, max_outer + 1))
    Z = np.zeros((n, max_outer))
    H = np.zeros((max_outer + 1, max_outer))
    V[:, 0] = r0 / beta
    e1 = np.zeros(max_outer + 1)
    e1[0] = beta
    ffom_prev = beta  # first-step bound ||r_1|| <= beta ||rhat_1||
    est_hist, ffom_hist, ks, reasons = [], [], [], []
    true_hist = [] if track_true else None
    rhat_hist = [] if (record or trace) else None
    rho_hist = [] if (record or trace) else None
    cycles = [] if record else None
    status = NOT_CONVERGED
    x = x0.copy()
    j_done = 0
    for j in range(max_outer):
        v = V[:, j]
        if level_steps:
            # preconditioner: an FGMRES run one level down (Section 5), to the tolerance the Eq. 5 bound asks for
            tau = tol * nb / ffom_prev if (c3 and np.isfinite(ffom_prev) and ffom_prev > 0.0) else 0.0
            child = fgmres(A, v, None, m=m, s=s, t=t, tol=tau, max_outer=level_steps[0], sketch_seed=sketch_seed,
                           zeta=zeta, sketch_kind=sketch_kind, cond_thr=cond_thr, c3=c3, outer_orth=outer_orth,
                           inner=inner, level_steps=level_steps[1:], _child=True)
            z = child.x
            ks.append(child.outer_iters)
            reasons.append(3 if child.status == CONVERGED else 1)
            if rho_hist is not None:
                rho_hist.append(child.est_hist[-1] if child.est_hist else float("inf"))
            if child.outer_iters == 0:  # the child's first cycle accepted no column: no correction
                status = BREAKDOWN
                break
        elif precond is None:
            scale = ffom_prev if (c3 and np.isfinite(ffom_prev)) else None
            cyc = sgmres_cycle(A if right_precond is None else A_in, v, S, m, t, cond_thr, bound_scale=scale,
                               bound_tol=tol * nb, inner=inner, A_inner=A_in, S_inner=S_in, record=record)
            z = cyc.z if right_precond is None else np.asarray(right_precond(cyc.z), dtype=np.float64)
            ks.append(cyc.k)
            reasons.append(cyc.reason)
            if rho_hist is not None:
                rho_hist.append(float(cyc.rho[-1]) if cyc.rho else float("inf"))
            if cycles is not None:
                cycles.append(cyc)
            if cyc.k == 0:
                status = BREAKDOWN
                break
        else:
            z = np.asarray(precond(v), dtype=np.float64)
        Z[:, j] = z
        w = A @ z
        if rhat_hist is not None:
            rhat_hist.append(float(np.linalg.norm(v - w)))
        if outer_orth == "mgs":  # Algorithm 1 as printed
            for i in range(j + 1):
                H[i, j] = V[:, i] @ w
                w = w - H[i, j] * V[:, i]
        elif outer_orth == "cgs2":
            Vj = V[:, : j + 1]
            h1 = Vj.T @ w
            w = w - Vj @ h1
            h2 = Vj.T @ w
            w = w - Vj @ h2
            H[: j + 1, j] = h1 + h2
        else:
            raise ValueError(outer_orth)
        H[j + 1, j] = np.linalg.norm(w)
        breakdown = H[j + 1, j] == 0.0
        if not breakdown:
            V[:, j + 1] = w / H[j + 1, j]
        Hj = H[: j + 2, : j + 1]
        rhs = e1[: j + 2]
        # FFOM residual, Eq. 4
        try:
            yF = np.linalg.solve(H[: j + 1, : j + 1], e1[: j + 1])
            ffom = float(H[j + 1, j] * abs(yF[-1]))
        except np.linalg.LinAlgError:
            yF = None
            ffom = np.inf
        if variant == "fgmres":
            y = np.linalg.lstsq(Hj, rhs, rcond=None)[0]
            est = float(np.linalg.norm(rhs - Hj @ y))
        elif variant == "ffom":
            if yF is None:
                status = BREAKDOWN
                break
            y = yF
            est = ffom
        else:
            raise ValueError(variant)
        est_hist.append(est / nb)
        ffom_hist.append(ffom / nb)
        j_done = j + 1
        if _child:
            # a lower level of a multi-level FGMRES: its estimate decides, and its last iterate is returned
            x = x0 + Z[:, : j + 1] @ y
            if est <= tol * nb or breakdown:
                status = CONVERGED
                break
            ffom_prev = ffom
            continue
        need_x = track_true or est <= tol * nb or breakdown or j + 1 == max_outer
        if need_x:
            x = x0 + Z[:, : j + 1] @ y
            rel_true = float(np.linalg.norm(b - A @ x)) / nb
            if true_hist is not None:
                true_hist.append(rel_true)
            if (est <= tol * nb and rel_true <= tol) or breakdown:
                status = CONVERGED
                break
        ffom_prev = ffom
    rel_true = float(np.linalg.norm(b - A @ x)) / nb
    res = FGMRESResult(x, status, j_done, rel_true, est_hist, ffom_hist, ks, reasons, true_hist, beta=beta,
                       rhat_hist=rhat_hist, rho_hist=rho_hist, cycles=cycles)
    if record:
        res.V = V[:, : j_done + 1]
        res.Z = Z[:, :j_done]
        res.H = H[: j_done + 1, :j_done]
    return res


def restarted(A, b: np.ndarray, x0: Optional[np.ndarray] = None, *, m: int, s: int, t: int, tol: float = 1e-8,
              max_outer: int = 50, sketch_seed: int = 1, zeta: int = 8, sketch_kind: str = "sparse_sign",
              cond_thr: float = 1e15, precond: Optional[Callable[[np.ndarray], np.ndarray]] = None):
    """Algorithm 2: restarting with a variable preconditioner; returns ``(x, [||r_j||/||b||], [||rhat_j||])``.

    With sGMRES as ``M_j`` the cycle is applied to the unit vector ``r_{j-1}/||r_{j-1}||`` and rescaled, so that
    ``z_j = M_j^{-1} r_{j-1}`` and ``rhat_j = r_{j-1} - A z_j``.
    """
    n = b.shape[0]
    nb = float(np.linalg.norm(b))
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    S = _sketch_for(n, s, zeta, sketch_seed, sketch_kind) if precond is None else None
    r = b - A @ x
    hist, rhat = [], []
    for _ in range(max_outer):
        nr = float(np.linalg.norm(r))
        if nr <= tol * nb:
            break
        if precond is None:
            z = nr * sgmres_cycle(A, r / nr, S, m, t, cond_thr).z
        else:
            z = np.asarray(precond(r), dtype=np.float64)
        rhat.append(float(np.linalg.norm(r - A @ z)))
        x = x + z
        r = b - A @ x
        hist.append(float(np.linalg.norm(r)) / nb)
    return x, hist, rhat
