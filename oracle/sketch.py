"""Sparse-sign subspace embedding ``S`` (oracle side).  TEST INFRASTRUCTURE ONLY.

The paper requires an epsilon-subspace embedding ``S in R^{s x n}``, ``m < s << n`` (Eq. 1, Section 1), drawn at
random, and uses in Section 4.1 the Clarkson-Woodruff sketch: one ``+-1`` per column in a uniformly random row.  This
library generalises it to the sparse-sign embedding with ``zeta`` nonzeros per column, each ``+-1/sqrt(zeta)`` in
``zeta`` *distinct* rows (``zeta = 1`` and unit scale is exactly the Clarkson-Woodruff sketch).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), written here from its published definition: the generator's state advances by the odd constant
``GAMMA`` and each output is the state passed through the 64-bit finaliser ``mix64``.  The k-th output (k = 0, 1,
...) of the stream started at state ``seed`` is therefore ``mix64(seed + (k+1)*GAMMA mod 2^64)``, which makes the
generator counter-based: any draw can be computed independently.

Draw layout (identical on the CUDA side, which implements the same definition independently):

* slot ``q = j*zeta + l`` for column ``j`` and nonzero ``l``;
* row candidate of attempt ``a`` (``0 <= a < 64``): ``h = draw(seed, 128*q + 2*a)``,
  ``row = ((h >> 32) * s) >> 32`` (multiply-shift range reduction of the top 32 bits);
  the first candidate not already used by slots ``0..l-1`` of the same column is taken; if all 64 attempts collide,
  the row after the last candidate (cyclically) that is still free is taken;
* sign: bit 63 of ``draw(seed, 128*q + 1)``; ``0`` means ``+``.
"""
from __future__ import annotations

import functools

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)
MAX_ATTEMPTS = 64


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser (published definition)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        return z ^ (z >> np.uint64(31))


def draw(seed: int, k) -> np.ndarray:
    """k-th output (0-based) of the SplitMix64 stream whose initial state is ``seed``."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (k + np.uint64(1)) * GAMMA
    return mix64(state)


def splitmix64_sequence(seed: int, count: int) -> np.ndarray:
    """First ``count`` outputs of SplitMix64 started at state ``seed`` (sequential form, for pinning ``draw``)."""
    out = np.empty(count, dtype=np.uint64)
    state = int(seed) & 0xFFFFFFFFFFFFFFFF
    for i in range(count):
        state = (state + int(GAMMA)) & 0xFFFFFFFFFFFFFFFF
        out[i] = mix64(np.uint64(state))
    return out


def _row_of(h: np.ndarray, s: int) -> np.ndarray:
    return ((h >> np.uint64(32)) * np.uint64(s)) >> np.uint64(32)


def sparse_sign_pattern(n: int, s: int, zeta: int, seed: int):
    """Rows ``int64[n, zeta]`` and signs ``int8[n, zeta]`` of the sparse-sign embedding (module docstring)."""
    if not (1 <= zeta <= s):
        raise ValueError("need 1 <= zeta <= s")
    j = np.arange(n, dtype=np.uint64)
    rows = np.empty((n, zeta), dtype=np.int64)
    signs = np.empty((n, zeta), dtype=np.int8)
    for l in range(zeta):
        q = j * np.uint64(zeta) + np.uint64(l)
        base = q * np.uint64(128)
        cand = _row_of(draw(seed, base), s).astype(np.int64)
        pending = np.any(rows[:, :l] == cand[:, None], axis=1) if l else np.zeros(n, dtype=bool)
        a = 1
        while pending.any() and a < MAX_ATTEMPTS:
            idx = np.nonzero(pending)[0]
            c2 = _row_of(draw(seed, base[idx] + np.uint64(2 * a)), s).astype(np.int64)
            cand[idx] = c2
            pending[idx] = np.any(rows[idx, :l] == c2[:, None], axis=1)
            a += 1
        for jj in np.nonzero(pending)[0]:  # all attempts collided: cyclic linear probe
            r = int(cand[jj])
            used = set(rows[jj, :l].tolist())
            while r in used:
                r = (r + 1) % s
            cand[jj] = r
        rows[:, l] = cand
        sb = draw(seed, base + np.uint64(1)) >> np.uint64(63)
        signs[:, l] = np.where(sb == 0, 1, -1).astype(np.int8)
    return rows, signs


@functools.lru_cache(maxsize=8)
def sketch_matrix(n: int, s: int, zeta: int = 8, seed: int = 1, kind: str = "sparse_sign"):
    """``S`` as a ``scipy.sparse.csr_matrix`` of shape ``(s, n)``.

    ``kind="sparse_sign"``: the embedding above, entries ``+-1/sqrt(zeta)``.
    ``kind="identity"``: ``S = I`` (requires ``s == n``), under which sGMRES reduces to GMRES.
    """
    import scipy.sparse as sp

    if kind == "identity":
        if s != n:
            raise ValueError("identity sketch needs s == n")
        return sp.identity(n, dtype=np.float64, format="csr")
    if kind != "sparse_sign":
        raise ValueError(kind)
    rows, signs = sparse_sign_pattern(n, s, zeta, seed)
    scale = 1.0 / np.sqrt(float(zeta))
    cols = np.repeat(np.arange(n, dtype=np.int64), zeta)
    vals = signs.reshape(-1).astype(np.float64) * scale
    return sp.csr_matrix((vals, (rows.reshape(-1), cols)), shape=(s, n))
