"""Textbook GMRES, used only to pin the oracle.  TEST INFRASTRUCTURE ONLY.

* :func:`gmres_brute` -- the GMRES iterate by its definition (Section 1: the correction minimises the residual norm
  over the Krylov space ``K_m(A, r_0)``): an orthonormal basis of ``[r0, A r0, ..., A^{m-1} r0]`` from a library QR,
  then a library least-squares solve.  Only for tiny, well-conditioned cases.
* :func:`gmres_restarted` -- restarted GMRES(m) (Saad & Schultz) with a modified Gram-Schmidt Arnoldi basis, for the
  qualitative comparisons of Section 2 (restarted GMRES stagnating while FGMRES converges).
"""
from __future__ import annotations

import numpy as np


def gmres_brute(A, b: np.ndarray, x0: np.ndarray, m: int) -> np.ndarray:
    r0 = b - A @ x0
    K = np.empty((b.shape[0], m))
    K[:, 0] = r0 / np.linalg.norm(r0)
    for i in range(1, m):
        K[:, i] = A @ K[:, i - 1]
        K[:, i] /= np.linalg.norm(K[:, i])
    Qk, _ = np.linalg.qr(K)
    AQ = np.column_stack([A @ Qk[:, i] for i in range(m)])
    y = np.linalg.lstsq(AQ, r0, rcond=None)[0]
    return x0 + Qk @ y


def gmres_restarted(A, b: np.ndarray, x0: np.ndarray, m: int, cycles: int, tol: float = 0.0):
    """GMRES(m); returns ``(x, [||r||/||b|| after each cycle])``."""
    n = b.shape[0]
    nb = np.linalg.norm(b)
    x = x0.copy()
    hist = []
    for _ in range(cycles):
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta <= tol * nb:
            break
        V = np.zeros((n, m + 1))
        H = np.zeros((m + 1, m))
        V[:, 0] = r / beta
        kk = m
        for j in range(m):
            w = A @ V[:, j]
            for i in range(j + 1):
                H[i, j] = V[:, i] @ w
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] == 0.0:
                kk = j + 1
                break
            V[:, j + 1] = w / H[j + 1, j]
        e1 = np.zeros(kk + 1)
        e1[0] = beta
        y = np.linalg.lstsq(H[: kk + 1, :kk], e1, rcond=None)[0]
        x = x + V[:, :kk] @ y
        hist.append(float(np.linalg.norm(b - A @ x) / nb))
    return x, hist
