"""Seeded synthetic inputs for the sketched-FGMRES solver (shared by the oracle, the tests and bench.py).

This module only *generates* problems ``A x = b`` (Section 1 states the method for a large sparse nonsymmetric
``A``); it contains none of the solver's arithmetic.  The paper's own matrices (SuiteSparse ``vas_stokes_1M``,
``ML_Geer``, ``NACA12`` ..., Section 4) are not available here; the workloads below stand in for them.

Generators
----------
* :func:`convdiff` -- upwind finite differences of ``-Laplace(u) + beta . grad(u)`` on the unit square/cube with
  homogeneous Dirichlet data, ``N`` interior points per side, ``h = 1/(N+1)``, lexicographic ordering (x fastest),
  every row scaled by ``h^2``.  Row ``i`` has diagonal ``2d + h*sum|beta_c|``; the upwind neighbour along axis ``c``
  (the ``-e_c`` side when ``beta_c >= 0``) gets ``-1 - h|beta_c|``, the downwind neighbour ``-1``; neighbours outside
  the domain are dropped.  2D 64^2 gives nnz 20,224, 3D 128^3 gives 14,581,760, 3D 64^3 gives 1,810,432.
* :func:`random_zipf` -- random nonsymmetric sparse matrix: row length ``L = clip(Zipf(1.5), 4, 256)`` including the
  diagonal, ``L-1`` distinct uniformly random off-diagonal columns, values ``N(0,1)``, diagonal set to ``1.2`` times
  the absolute off-diagonal row sum (strictly diagonally dominant, hence nonsingular).
* :func:`rhs` -- right-hand sides ``N(0,1)`` or ``U(-1,1)``.
* :func:`convdiff_batch` -- a batch of independent 2D convection-diffusion systems with grid sides uniform in
  ``[nmin, nmax]`` and ``beta ~ U(0, beta_max)^2`` per system, returned as one block-diagonal CSR matrix
  (:func:`block_diag`) with the systems' orders in ``CSR.sys_n``; :func:`batch_rhs` draws ``nrhs`` right-hand sides
  per system in problem order (system-major, then right-hand side).

Every generator draws from ``numpy.random.default_rng([seed, stream])`` with a fixed stream tag per purpose, so the
same ``seed`` gives independent streams for ``A``, ``b``, ``x*`` and batch parameters.

CSR arrays are returned as ``(row_ptr int64[n+1], col int32[nnz], val float64[nnz])`` with sorted column indices.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Tuple

import numpy as np

# stream tags for default_rng([seed, tag])
STREAM_MATRIX = 0
STREAM_RHS = 1
STREAM_XSTAR = 2
STREAM_BATCH = 3
STREAM_SAMPLE = 4


@dataclasses.dataclass
class CSR:
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[nnz]
    val: np.ndarray  # float64[nnz]
    sys_n: Optional[np.ndarray] = None  # orders of the diagonal blocks of a batch (None: one system)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))


def convdiff(N: int, beta, d: int | None = None) -> CSR:
    """Upwind convection-diffusion matrix on an ``N^d`` interior grid (see module docstring)."""
    beta = np.asarray(beta, dtype=np.float64)
    if d is None:
        d = beta.size
    assert beta.size == d and d in (1, 2, 3) and N >= 1
    n = N ** d
    h = 1.0 / (N + 1)
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for _ in range(d):  # x fastest
        coords.append(rem % N)
        rem //= N
    strides = [N ** c for c in range(d)]
    # neighbour slots in increasing column order: -e_{d-1},...,-e_0, diag, +e_0,...,+e_{d-1}
    offs, vals, valid = [], [], []
    for c in reversed(range(d)):
        up = beta[c] >= 0.0  # -e_c side is upwind
        offs.append(-strides[c])
        vals.append(-1.0 - h * abs(beta[c]) if up else -1.0)
        valid.append(coords[c] > 0)
    offs.append(0)
    vals.append(2.0 * d + h * float(np.abs(beta).sum()))
    valid.append(np.ones(n, dtype=bool))
    for c in range(d):
        up = beta[c] < 0.0  # +e_c side is upwind
        offs.append(strides[c])
        vals.append(-1.0 - h * abs(beta[c]) if up else -1.0)
        valid.append(coords[c] < N - 1)
    k = len(offs)
    mask = np.stack(valid, axis=1)  # (n, k)
    cols = idx[:, None] + np.asarray(offs, dtype=np.int64)[None, :]
    v = np.broadcast_to(np.asarray(vals, dtype=np.float64)[None, :], (n, k))
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n, row_ptr, cols[mask].astype(np.int32), np.ascontiguousarray(v[mask]))


def random_zipf(n: int, seed: int = 0, a: float = 1.5, lmin: int = 4, lmax: int = 256,
                dominance: float = 1.2) -> CSR:
    """Random nonsymmetric sparse matrix with Zipf row lengths (see module docstring)."""
    rng = np.random.default_rng([seed, STREAM_MATRIX])
    lmax = min(lmax, n)
    lmin = min(lmin, lmax)
    L = np.clip(rng.zipf(a, size=n), lmin, lmax).astype(np.int64)
    noff = L - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), noff)
    # uniform over the n-1 off-diagonal columns of each row
    c = rng.integers(0, n - 1, size=rows.size, dtype=np.int64)
    c += (c >= rows)
    while True:
        key = rows * n + c
        order = np.argsort(key, kind="stable")
        key = key[order]
        rows = rows[order]
        c = c[order]
        dup = np.zeros(key.size, dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0:
            break
        r = rng.integers(0, n - 1, size=nd, dtype=np.int64)
        c[dup] = r + (r >= rows[dup])
    offv = rng.standard_normal(rows.size)
    absum = np.bincount(rows, weights=np.abs(offv), minlength=n)
    diag = dominance * absum
    # merge the diagonal into the sorted column lists
    all_rows = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    all_cols = np.concatenate([c, np.arange(n, dtype=np.int64)])
    all_vals = np.concatenate([offv, diag])
    order = np.lexsort((all_cols, all_rows))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(L, out=row_ptr[1:])
    return CSR(n, row_ptr, all_cols[order].astype(np.int32), all_vals[order])


def rhs(n: int, seed: int = 0, dist: str = "normal", stream: int = STREAM_RHS, nrhs: int | None = None) -> np.ndarray:
    """Right-hand side(s): ``dist`` is ``"normal"`` (N(0,1)) or ``"uniform"`` (U(-1,1)).  Shape ``(n,)`` or ``(nrhs, n)``."""
    rng = np.random.default_rng([seed, stream])
    shape = (n,) if nrhs is None else (nrhs, n)
    if dist == "normal":
        return rng.standard_normal(shape)
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, shape)
    raise ValueError(dist)


def block_diag(mats: List[CSR]) -> CSR:
    """The block-diagonal matrix diag(A_0, A_1, ...) in CSR (global column indices), with ``sys_n`` set."""
    sys_n = np.asarray([A.n for A in mats], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(sys_n)])
    noff = np.concatenate([[0], np.cumsum([A.nnz for A in mats])])
    row_ptr = np.concatenate([[0]] + [A.row_ptr[1:] + noff[q] for q, A in enumerate(mats)]).astype(np.int64)
    col = np.concatenate([A.col.astype(np.int64) + off[q] for q, A in enumerate(mats)]).astype(np.int32)
    val = np.concatenate([A.val for A in mats])
    return CSR(int(off[-1]), row_ptr, col, val, sys_n)


def split_blocks(A: CSR) -> List[CSR]:
    """The diagonal blocks of a block-diagonal CSR built by :func:`block_diag` (local column indices)."""
    out = []
    off = 0
    for nq in A.sys_n:
        nq = int(nq)
        a, e = int(A.row_ptr[off]), int(A.row_ptr[off + nq])
        out.append(CSR(nq, A.row_ptr[off:off + nq + 1] - a, (A.col[a:e].astype(np.int64) - off).astype(np.int32),
                       A.val[a:e].copy()))
        off += nq
    return out


def convdiff_batch(nsys: int, nmin: int = 32, nmax: int = 512, beta_max: float = 50.0, seed: int = 0) -> CSR:
    """Batch of 2D upwind convection-diffusion systems (see module docstring), block-diagonal CSR."""
    rng = np.random.default_rng([seed, STREAM_BATCH])
    sides = rng.integers(nmin, nmax + 1, size=nsys)
    betas = rng.uniform(0.0, beta_max, size=(nsys, 2))
    return block_diag([convdiff(int(N), betas[q]) for q, N in enumerate(sides)])


def batch_rhs(sys_n, nrhs: int, seed: int = 0, dist: str = "normal") -> np.ndarray:
    """``nrhs`` right-hand sides per system in problem order: problem ``p = q * nrhs + r`` occupies the ``sys_n[q]``
    entries starting at ``nrhs * off_q + r * sys_n[q]``; one N(0,1) (or U(-1,1)) draw of the whole vector."""
    total = int(np.sum(sys_n)) * nrhs
    return rhs(total, seed=seed, dist=dist, stream=STREAM_RHS)


def problem_slices(sys_n, nrhs: int):
    """(system, start, length) of every problem of a batch, in problem order."""
    out = []
    off = 0
    for q, nq in enumerate(sys_n):
        nq = int(nq)
        for r in range(nrhs):
            out.append((q, nrhs * off + r * nq, nq))
        off += nq
    return out


@dataclasses.dataclass
class Config:
    """One solver workload: matrix recipe, right-hand side recipe and sGMRES/FGMRES parameters.

    ``m`` is the inner sGMRES basis size (the paper's ``k_max``), ``t`` the Arnoldi truncation depth, ``s`` the
    sketch rows, ``zeta`` nonzeros per sketch column, ``sketch_seed`` the embedding's seed.
    """
    name: str
    matrix: Tuple
    rhs_dist: str
    m: int
    t: int
    s: int
    zeta: int = 8
    sketch_seed: int = 1
    tol: float = 1e-8
    max_outer: int = 50
    seed: int = 0
    nrhs: int = 1
    precision: str = "fp64"

    def build_matrix(self) -> CSR:
        kind = self.matrix[0]
        if kind == "convdiff":
            _, N, beta = self.matrix
            return convdiff(N, beta)
        if kind == "zipf":
            _, n = self.matrix
            return random_zipf(n, seed=self.seed)
        if kind == "convdiff_batch":
            _, nsys, nmin, nmax, beta_max = self.matrix
            return convdiff_batch(nsys, nmin, nmax, beta_max, seed=self.seed)
        raise ValueError(kind)

    def build_rhs(self, n: int) -> np.ndarray:
        """Right-hand side(s): ``(n,)`` for one system and one right-hand side, else ``nrhs * n`` values in problem
        order."""
        if self.matrix[0] == "convdiff_batch" or self.nrhs > 1:
            return batch_rhs([n] if self.matrix[0] != "convdiff_batch" else self.build_matrix().sys_n, self.nrhs,
                             seed=self.seed, dist=self.rhs_dist)
        return rhs(n, seed=self.seed, dist=self.rhs_dist)


CONFIGS: Dict[str, Config] = {
    # 2D convection-diffusion 64x64, beta=(20,10); m=30, t=2, s=120; at most 20 outer iterations
    "cd2d_64": Config("cd2d_64", ("convdiff", 64, (20.0, 10.0)), "normal", m=30, t=2, s=120, max_outer=20),
    # 3D convection-diffusion 128^3, beta=(50,30,10); m=100, t=2, s=400
    "cd3d_128": Config("cd3d_128", ("convdiff", 128, (50.0, 30.0, 10.0)), "normal", m=100, t=2, s=400),
    # random Zipf(1.5) rows, n = 2,000,000; m=60, t=4, s=240
    "zipf_2m": Config("zipf_2m", ("zipf", 2_000_000), "uniform", m=60, t=4, s=240),
    # 3D convection-diffusion 64^3 (adjoint workload); m=50, t=2, s=200
    "cd3d_64": Config("cd3d_64", ("convdiff", 64, (50.0, 30.0, 10.0)), "normal", m=50, t=2, s=200),
    # batch: 512 2D convection-diffusion systems, sides U{32..512}, beta ~ U(0,50)^2, 4 right-hand sides each;
    # m=40, t=2, s=160, FP32 inner cycles with the FP64 outer FGMRES
    # (the 512^2 systems with weak convection need ~45 outer iterations, hence max_outer = 60)
    "batch_512": Config("batch_512", ("convdiff_batch", 512, 32, 512, 50.0), "normal", m=40, t=2, s=160, nrhs=4,
                        precision="fp32", max_outer=60),
    # small batch of the same recipe (sides 16..48, 12 systems, 3 right-hand sides) for oracle parity
    "batch_small": Config("batch_small", ("convdiff_batch", 12, 16, 48, 50.0), "normal", m=40, t=2, s=160, nrhs=3),
}
