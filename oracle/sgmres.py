"""One sketched-GMRES cycle, used as the variable preconditioner of FGMRES (oracle side).  TEST INFRASTRUCTURE ONLY.

Follows Section 3 (and Eq. 3 of Section 1): given a unit vector ``v``, build a non-orthogonal basis ``B_k`` of the
Krylov space ``K_k(A, v)`` by truncated Arnoldi (Section 4.1: each new vector is orthogonalised against the previous
``t`` basis vectors only; ``t = 0`` gives a normalised power basis), and return

    z = B_k y_k,      y_k = argmin_y || S v - S A B_k y ||          (Section 3; Eq. 3 with r_0 = v, x_0 = 0)

The sketched least-squares problem is solved through a QR factorisation ``Q_k R_k = S A B_k`` updated one column at
a time by classical Gram-Schmidt with one reorthogonalisation pass (Section 3, C2).  ``k`` is as large as possible
subject to

* C1: ``k <= k_max`` (here ``m``);
* C2: ``cond(S A B_k) <= threshold`` (1e15), evaluated on ``R_k`` through the proxy ``max|r_ll| / min|r_ll|``; the
  column that pushes the proxy above the threshold is dropped;
* C3: the bound of Eq. 5 predicts that the outer FGMRES residual meets the tolerance:
  ``bound_scale * rho_i <= bound_tol``, where ``rho_i = ||S v - S A B_i y_i||`` is the sketched residual of the
  inner problem and ``bound_scale`` is the FFOM residual of the previous outer step (``beta`` at the first step).

An exact breakdown ``eta_i = 0`` of the truncated Arnoldi recurrence ends the cycle with ``k = i``.

Precision (``inner``): ``"fp64"``; ``"fp32"`` (matrix values, basis, dot products, sketch and their accumulation in
FP32, QR and least squares in FP64); ``"bf16"`` (as fp32 but every stored basis vector rounded to BF16).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.linalg as sla

from .lowprec import INNER_DTYPES, store

# reasons a cycle stopped
STOP_C1 = 1  # k reached m
STOP_C2 = 2  # condition-number proxy above threshold (column dropped)
STOP_C3 = 3  # Eq. 5 bound met the tolerance
STOP_BREAKDOWN = 4  # eta_i == 0: Krylov space invariant
STOP_DEGENERATE = 5  # first sketched column is zero: no basis at all (k = 0)


@dataclasses.dataclass
class CycleResult:
    z: np.ndarray  # FP64 correction B_k y_k
    k: int
    y: np.ndarray
    reason: int
    rho: List[float]  # sketched residual after each accepted column
    kappa: List[float]  # condition proxy after each column tried
    basis: Optional[List[np.ndarray]] = None  # b_1..b_{k} (inner storage precision) if recorded
    sab: Optional[np.ndarray] = None  # S A B_k (FP64, s x k) if recorded
    R: Optional[np.ndarray] = None
    c0: Optional[np.ndarray] = None
    h: Optional[List[np.ndarray]] = None  # truncated-Arnoldi coefficients per step
    eta: Optional[List[float]] = None


def sgmres_cycle(A, v: np.ndarray, S, m: int, t: int, cond_thr: float = 1e15,
                 bound_scale: Optional[float] = None, bound_tol: float = 0.0,
                 inner: str = "fp64", A_inner=None, S_inner=None, record: bool = False) -> CycleResult:
    """Approximate ``A z = v`` by one sGMRES cycle with zero initial guess (Algorithm 1 with Section 3).

    ``A`` and ``S`` are scipy sparse FP64 matrices; ``A_inner``/``S_inner`` are their copies in the inner
    precision (built here when omitted).  ``bound_scale=None`` disables C3.
    """
    dt = INNER_DTYPES[inner]
    if A_inner is None:
        A_inner = A if dt == np.float64 else A.astype(dt)
    if S_inner is None:
        S_inner = S if dt == np.float64 else S.astype(dt)
    s = S.shape[0]

    b1 = store(v, inner)
    basis = [b1]
    c0 = np.asarray(S_inner @ b1, dtype=np.float64)  # S v (sketched in the inner precision)
    Q = np.zeros((s, m))
    R = np.zeros((m, m))
    C = np.zeros((s, m))  # S A B
    rho: List[float] = []
    kappa: List[float] = []
    hs: List[np.ndarray] = []
    etas: List[float] = []
    k = 0
    reason = STOP_C1
    for i in range(m):  # paper index i+1
        w = A_inner @ basis[i]  # A b_i (inner precision)
        c = np.asarray(S_inner @ w, dtype=np.float64)  # S A b_i, one sketch per iteration
        # Gram-Schmidt with one reorthogonalisation pass against q_1..q_{i-1}
        Qi = Q[:, :i]
        a1 = Qi.T @ c
        p = c - Qi @ a1
        a2 = Qi.T @ p
        p = p - Qi @ a2
        R[:i, i] = a1 + a2
        R[i, i] = np.linalg.norm(p)
        d = np.abs(np.diag(R)[: i + 1])
        kap = float(d.max() / d.min()) if d.min() > 0.0 else np.inf
        kappa.append(kap)
        if kap > cond_thr:  # C2: drop column i+1, keep B_i
            k = i
            reason = STOP_C2 if i > 0 else STOP_DEGENERATE
            break
        Q[:, i] = p / R[i, i]
        C[:, i] = c
        # sketched residual of the least-squares problem over the first i+1 columns
        yi = sla.solve_triangular(R[: i + 1, : i + 1], Q[:, : i + 1].T @ c0)
        rho_i = float(np.linalg.norm(c0 - C[:, : i + 1] @ yi))
        rho.append(rho_i)
        k = i + 1
        if bound_scale is not None and bound_scale * rho_i <= bound_tol:  # C3
            reason = STOP_C3
            break
        if k == m:  # C1
            reason = STOP_C1
            break
        # truncated Arnoldi: orthogonalise against the last t basis vectors (classical GS form)
        lo = max(0, i - t + 1)
        h = np.array([np.dot(basis[l], w) for l in range(lo, i + 1)], dtype=dt)
        u = w.copy()
        for l, hl in zip(range(lo, i + 1), h):
            u = u - hl * basis[l]
        eta = dt(np.linalg.norm(u))
        hs.append(h)
        etas.append(float(eta))
        if eta == 0.0:
            reason = STOP_BREAKDOWN
            break
        basis.append(store(u / eta, inner))
    if k == 0:
        y = np.zeros(0)
        z = np.zeros(v.shape[0])
    else:
        y = sla.solve_triangular(R[:k, :k], Q[:, :k].T @ c0)
        z = np.zeros(v.shape[0])
        for l in range(k):
            z += y[l] * basis[l].astype(np.float64)
    res = CycleResult(z=z, k=k, y=y, reason=reason, rho=rho, kappa=kappa)
    if record:
        res.basis = list(basis)  # every vector formed: b_1..b_k, plus b_{k+1} when C2 dropped column k+1
        res.sab = C[:, :k].copy()
        res.R = R[:k, :k].copy()
        res.c0 = c0
        res.h = hs
        res.eta = etas
    return res
