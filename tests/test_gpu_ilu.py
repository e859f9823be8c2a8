"""GPU parity of ILU(0) right preconditioning in a multicolour order (the "-p" runs of Section 4, Table 1) against the
oracle (``oracle.ilu``: colouring, ILU(0), triangular solves; ``oracle.fgmres(right_precond=...)``) on the same
seeded inputs.

* The colouring (integer work) equals the oracle's row for row: a greedy colouring of the pattern of A + A^T in the
  natural order; red-black for the 5- and 7-point stencils, many colours for the random Zipf pattern.
* The ILU(0) factors of the colour-permuted matrix agree with the oracle's to 1e-13 relative to the largest entry
  (the same eliminations in the same order; FP64 rounding of fused multiply-adds apart), also after new values of A.
* Right-preconditioned solves: both reach 1e-8 (recomputed), outer counts within 1, the same inner lengths for every
  cycle but the last, and the per-step estimates within 1e-6 relative while both run.
* Uses the preconditioner does not support are refused.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import fgmres as ofg
from oracle import ilu as oilu

from gpu_common import dev_vec, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _solver(A, **opt):
    from paper_2506_18408_gb300 import Solver

    return Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=1, **opt)


def _oracle_mc(As):
    """The oracle's multicolour ILU(0): colours, permutation, factors of P A P^T, and u -> M^{-1} u."""
    perm, colours, starts = oilu.colouring(As)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    Pm = As[perm][:, perm].tocsr()
    L, U = oilu.ilu0(Pm)

    def apply(u):
        z = oilu.ilu0_solve(L, U, u[perm])
        out = np.empty_like(z)
        out[perm] = z
        return out

    return colours, inv, L, U, apply


def _factor_values_in_a_order(A, inv, L, U):
    """For every stored entry (i, j) of A: the entry (p(i), p(j)) of L (strictly below the diagonal) or U."""
    LU = (sp.csr_matrix(L) - sp.identity(A.n, format="csr") + sp.csr_matrix(U)).tocsr()
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    r, c = inv[rows], inv[A.col]
    return np.asarray(LU[r, c]).ravel()


CASES = [
    ("cd3d_12", lambda: workloads.convdiff(12, (50.0, 30.0, 10.0))),
    ("cd2d_32", lambda: workloads.convdiff(32, (20.0, 10.0))),
    ("zipf_3000", lambda: workloads.random_zipf(3000, seed=2)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_colouring_and_factors_match_oracle(name, make):
    A = make()
    As = A.to_scipy().tocsr()
    sv = _solver(A)
    colour, ncol, lu = sv.precond_info()
    colours, inv, L, U, _ = _oracle_mc(As)
    assert np.array_equal(colour.astype(np.int64), colours)
    assert ncol == int(colours.max()) + 1
    if name != "zipf_3000":
        assert ncol == 2  # red-black for the stencils
    ref = _factor_values_in_a_order(A, inv, L, U)
    scale = np.abs(ref).max()
    assert np.abs(lu - ref).max() <= 1e-13 * scale, (name, np.abs(lu - ref).max() / scale)
    # new values of A: the factors follow
    A2 = workloads.convdiff(12, (5.0, 3.0, 1.0)) if name == "cd3d_12" else None
    if A2 is not None:
        sv.update_values(A2.val)
        _, _, lu2 = sv.precond_info()
        _, inv2, L2, U2, _ = _oracle_mc(A2.to_scipy().tocsr())
        ref2 = _factor_values_in_a_order(A2, inv2, L2, U2)
        assert np.abs(lu2 - ref2).max() <= 1e-13 * np.abs(ref2).max()
    sv.close()


SOLVES = [
    ("cd2d_48", lambda: workloads.convdiff(48, (20.0, 10.0)), 40, 160, 2),
    ("cd3d_16", lambda: workloads.convdiff(16, (50.0, 30.0, 10.0)), 40, 160, 2),
    ("cd3d_16_t0", lambda: workloads.convdiff(16, (50.0, 30.0, 10.0)), 30, 120, 0),
]


@pytest.mark.parametrize("name,make,m,s,t", SOLVES, ids=[c[0] for c in SOLVES])
def test_preconditioned_solve_against_oracle(name, make, m, s, t):
    A = make()
    As = A.to_scipy().tocsr()
    b = workloads.rhs(A.n, seed=0)
    sv = _solver(A, max_outer=50, precond=1)
    x, info = sv.solve(dev_vec(b), m=m, s=s, k=t, tol=1e-8)
    _, _, _, _, apply = _oracle_mc(As)
    ref = ofg.fgmres(As, b, m=m, s=s, t=t, tol=1e-8, max_outer=50, right_precond=apply)
    plain = ofg.fgmres(As, b, m=m, s=s, t=t, tol=1e-8, max_outer=50)
    rel = float(np.linalg.norm(b - As @ x.cpu().numpy()) / np.linalg.norm(b))
    print(f"{name}: GPU outer {info['outer_iters']} inner {info['total_inner']} | oracle {ref.outer_iters} "
          f"{sum(ref.inner_k)} | unpreconditioned oracle {plain.outer_iters} {sum(plain.inner_k)}")
    assert info["status"] == 0 and ref.status == ofg.CONVERGED
    assert rel <= 1e-8 and ref.rel_res_true <= 1e-8
    assert abs(info["outer_iters"] - ref.outer_iters) <= 1
    common = min(len(info["inner_k"]), len(ref.inner_k)) - 1
    assert info["inner_k"][:common] == ref.inner_k[:common]
    if t > 0:  # the power basis (t = 0) amplifies rounding differences; counts and convergence only
        est = info["res_est"]
        for j in range(min(len(est), len(ref.est_hist)) - 1):
            assert abs(est[j] - ref.est_hist[j]) <= 1e-6 * ref.est_hist[j], (j, est[j], ref.est_hist[j])
    assert sum(ref.inner_k) < sum(plain.inner_k)  # the preconditioner pays


def test_unsupported_uses_are_refused():
    from paper_2506_18408_gb300 import sfgmres as py

    A = workloads.convdiff(10, (1.0, 1.0))
    b = dev_vec(workloads.rhs(A.n, seed=0))
    sv = _solver(A, precond=1, precision="fp32")
    with pytest.raises(py.SFGMRESError) as e:
        sv.solve(b, m=10, s=40, k=2)
    assert e.value.code == py.ERR_INVALID_ARG
    sv.set("precision", "fp64")
    with pytest.raises(py.SFGMRESError) as e:
        sv.solve(b, m=10, s=40, k=2, transpose=True)
    assert e.value.code == py.ERR_INVALID_ARG
    x, info = sv.solve(b, m=10, s=40, k=2)  # the supported use still works
    assert info["status"] == 0
    # a matrix without one of its diagonal entries
    keep = ~((np.repeat(np.arange(A.n), np.diff(A.row_ptr)) == 5) & (A.col == 5))
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))[keep]
    rp = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=A.n))]).astype(np.int64)
    from paper_2506_18408_gb300 import Solver

    sv2 = Solver(A.n, rp, A.col[keep], A.val[keep], sketch_seed=1, precond=1)
    with pytest.raises(py.SFGMRESError) as e:
        sv2.solve(b, m=10, s=40, k=2)
    assert e.value.code == py.ERR_INVALID_ARG
