"""Zero-fill incomplete LU (ILU(0)), the preconditioner of the paper's "-p" experiments (Section 4, Table 1).
TEST INFRASTRUCTURE ONLY.

:func:`ilu0` factors a sparse A into a unit lower triangular L and an upper triangular U whose nonzeros lie in the
pattern of A, by Gaussian elimination in row order (the IKJ form) in which every update that would create an entry
outside that pattern is dropped.  Consequently (L U)_ij = A_ij for every (i, j) in the pattern of A, and when the
pattern of A admits no fill (a tridiagonal matrix, for instance) L U is the exact LU factorisation without pivoting.
:func:`ilu0_solve` applies M^{-1} = (L U)^{-1} by forward and back substitution.  :func:`colouring` orders the
rows colour by colour (a greedy colouring of the symmetrised pattern: no two coupled rows share a colour), so that
ILU(0) of the symmetrically permuted matrix P A P^T has diagonal colour blocks in both factors and each colour's rows
of a triangular solve are independent of one another.  Plain Python loops over the rows: for the small matrices of
the pins only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def ilu0(A):
    """Returns ``(L, U)`` as SciPy CSR matrices: L unit lower triangular (its unit diagonal stored), U upper
    triangular, both with their nonzeros in the pattern of A.  Raises ``ZeroDivisionError`` on a zero pivot."""
    A = sp.csr_matrix(A, dtype=np.float64)
    A.sort_indices()
    n = A.shape[0]
    rows = []
    for i in range(n):
        a, e = A.indptr[i], A.indptr[i + 1]
        rows.append(dict(zip(A.indices[a:e].tolist(), A.data[a:e].tolist())))
    for i in range(n):
        ri = rows[i]
        for k in sorted(c for c in ri if c < i):  # eliminate with rows k < i in increasing order
            ukk = rows[k].get(k, 0.0)
            if ukk == 0.0:
                raise ZeroDivisionError(f"zero pivot in row {k}")
            lik = ri[k] / ukk
            ri[k] = lik
            for j, ukj in rows[k].items():
                if j > k and j in ri:  # updates outside the pattern of A are dropped
                    ri[j] -= lik * ukj
    li, lj, lv, ui, uj, uv = [], [], [], [], [], []
    for i, ri in enumerate(rows):
        li.append(i), lj.append(i), lv.append(1.0)
        for j, v in ri.items():
            if j < i:
                li.append(i), lj.append(j), lv.append(v)
            else:
                ui.append(i), uj.append(j), uv.append(v)
    L = sp.csr_matrix((lv, (li, lj)), shape=(n, n))
    U = sp.csr_matrix((uv, (ui, uj)), shape=(n, n))
    return L, U


def ilu0_solve(L, U, v: np.ndarray) -> np.ndarray:
    """z = (L U)^{-1} v: forward substitution with the unit lower L, then back substitution with U."""
    n = v.shape[0]
    L = sp.csr_matrix(L)
    U = sp.csr_matrix(U)
    y = np.array(v, dtype=np.float64)
    for i in range(n):
        a, e = L.indptr[i], L.indptr[i + 1]
        for p in range(a, e):
            j = L.indices[p]
            if j < i:
                y[i] -= L.data[p] * y[j]
    z = y
    for i in range(n - 1, -1, -1):
        a, e = U.indptr[i], U.indptr[i + 1]
        d = 0.0
        for p in range(a, e):
            j = U.indices[p]
            if j > i:
                z[i] -= U.data[p] * z[j]
            elif j == i:
                d = U.data[p]
        if d == 0.0:
            raise ZeroDivisionError(f"zero diagonal of U in row {i}")
        z[i] /= d
    return z


def colouring(A):
    """Greedy colouring of the pattern of A + A^T (every stored entry of A is an edge, whatever its value; each row, in natural order, takes the smallest colour not used by
    an already coloured neighbour).  Returns ``(perm, colours, starts)``: ``perm`` lists the rows colour by colour
    (natural order within a colour), ``colours[i]`` is row i's colour, and colour c occupies positions
    ``starts[c] .. starts[c + 1]`` of ``perm``."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    P = A.copy()
    P.data = np.ones_like(P.data)  # the stored pattern alone: a pair a_ij = -a_ji must not cancel in A + A^T
    G = (P + P.T).tocsr()
    colours = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        used = {int(colours[j]) for j in G.indices[G.indptr[i]:G.indptr[i + 1]] if j != i and colours[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colours[i] = c
    nc = int(colours.max()) + 1 if n else 0
    perm = np.concatenate([np.flatnonzero(colours == c) for c in range(nc)]) if n else np.zeros(0, np.int64)
    starts = np.concatenate([[0], np.cumsum([np.count_nonzero(colours == c) for c in range(nc)])])
    return perm, colours, starts
