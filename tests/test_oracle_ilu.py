"""Pins for the oracle's zero-fill incomplete LU (the ILU(0) preconditioner of the paper's "-p" runs)."""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

import workloads
from oracle import ilu


def _pattern(M):
    M = sp.coo_matrix(M)
    return set(zip(M.row.tolist(), M.col.tolist()))


def test_tridiagonal_has_no_fill_so_ilu0_is_the_exact_lu():
    rng = np.random.default_rng(0)
    n = 40
    A = sp.diags([rng.uniform(-1, 1, n - 1), rng.uniform(4, 5, n), rng.uniform(-1, 1, n - 1)], [-1, 0, 1]).tocsr()
    L, U = ilu.ilu0(A)
    np.testing.assert_allclose((L @ U).toarray(), A.toarray(), rtol=0, atol=1e-14)
    # against the textbook LU without pivoting (Doolittle), written out densely
    D = A.toarray()
    Ld, Ud = np.eye(n), D.copy()
    for k in range(n - 1):
        for i in range(k + 1, n):
            Ld[i, k] = Ud[i, k] / Ud[k, k]
            Ud[i, k:] -= Ld[i, k] * Ud[k, k:]
    np.testing.assert_allclose(L.toarray(), Ld, rtol=0, atol=1e-14)
    np.testing.assert_allclose(U.toarray(), np.triu(Ud), rtol=0, atol=1e-13)
    v = rng.standard_normal(n)
    np.testing.assert_allclose(ilu.ilu0_solve(L, U, v), np.linalg.solve(D, v), rtol=1e-12, atol=1e-12)


def test_product_matches_a_on_its_pattern_and_factors_stay_in_it():
    A = workloads.convdiff(12, (20.0, 10.0)).to_scipy().tocsr()  # 5-point upwind: fill would appear in exact LU
    L, U = ilu.ilu0(A)
    pa = _pattern(A)
    assert _pattern(sp.tril(L, -1)) <= pa and _pattern(U) <= pa
    assert np.all(sp.triu(L, 1).toarray() == 0) and np.all(sp.tril(U, -1).toarray() == 0)
    np.testing.assert_array_equal(L.diagonal(), np.ones(A.shape[0]))
    P = (L @ U).tocsr()
    Ad = A.toarray()
    for i, j in pa:
        assert abs(P[i, j] - Ad[i, j]) <= 1e-12 * max(1.0, abs(Ad[i, j])), (i, j)
    # the exact LU does fill in: ILU(0) drops those entries, so L U differs from A off the pattern
    assert np.abs((P - A).toarray()).max() > 1e-6
    Lx, Ux = sla.lu(Ad, permute_l=False)[1:]
    assert np.count_nonzero(np.abs(Ux) > 1e-14) > U.nnz


def test_solve_inverts_the_product_and_diagonal_special_case():
    rng = np.random.default_rng(1)
    A = workloads.convdiff(10, (5.0, 3.0)).to_scipy().tocsr()
    L, U = ilu.ilu0(A)
    v = rng.standard_normal(A.shape[0])
    z = ilu.ilu0_solve(L, U, v)
    np.testing.assert_allclose((L @ U) @ z, v, rtol=0, atol=1e-12 * np.abs(v).max())
    d = rng.uniform(1, 2, 25)
    L2, U2 = ilu.ilu0(sp.diags(d).tocsr())
    np.testing.assert_array_equal(L2.toarray(), np.eye(25))
    np.testing.assert_array_equal(U2.diagonal(), d)
    np.testing.assert_allclose(ilu.ilu0_solve(L2, U2, v[:25]), v[:25] / d, rtol=1e-15)


def test_preconditioned_operator_is_much_better_conditioned():
    """M^{-1} A (M = L U from ILU(0)) is far better conditioned than A scaled by its diagonal on the convection-
    diffusion matrices (the reason for the paper's preconditioned runs): measured 2-5 against 23-48 for the 2D
    100-point matrices below, so a factor of 4 is a safe margin."""
    for beta in ((20.0, 10.0), (5.0, 3.0), (0.0, 0.0), (50.0, 30.0)):
        A = workloads.convdiff(10, beta).to_scipy().tocsr()
        L, U = ilu.ilu0(A)
        n = A.shape[0]
        Minv_A = np.column_stack([ilu.ilu0_solve(L, U, A[:, [k]].toarray().ravel()) for k in range(n)])
        Dinv_A = A.toarray() / A.diagonal()[:, None]
        assert np.linalg.cond(Minv_A) < 0.25 * np.linalg.cond(Dinv_A), beta


def test_right_preconditioned_fgmres_special_cases_and_ilu0_gain():
    """FGMRES with the inner sGMRES cycles on A M^{-1} and z_j = M^{-1} (their result): with M = I it is the
    unpreconditioned run bit for bit; with M = A (exact solves) A M^{-1} = I, so one outer step with a one-column
    cycle solves the system to rounding; with M = ILU(0) it converges in far fewer outer and inner steps on the
    convection-diffusion matrix (measured 5 outer / 36 inner against 13 / 122)."""
    import scipy.sparse.linalg as spl
    from oracle import fgmres as ofg

    A = workloads.convdiff(32, (20.0, 10.0)).to_scipy().tocsr()
    b = workloads.rhs(A.shape[0], seed=0)
    kw = dict(m=10, s=40, t=2, tol=1e-8, max_outer=60)
    plain = ofg.fgmres(A, b, None, **kw)
    ident = ofg.fgmres(A, b, None, right_precond=lambda u: np.array(u, dtype=np.float64), **kw)
    assert ident.est_hist == plain.est_hist and ident.inner_k == plain.inner_k
    Ac = A.tocsc()
    exact = ofg.fgmres(A, b, None, right_precond=lambda u: spl.spsolve(Ac, u), **kw)
    assert exact.status == 0 and exact.outer_iters == 1 and exact.inner_k == [1]
    assert exact.rel_res_true <= 1e-14
    L, U = ilu.ilu0(A)
    pre = ofg.fgmres(A, b, None, right_precond=lambda u: ilu.ilu0_solve(L, U, u), **kw)
    assert plain.status == 0 and pre.status == 0 and pre.rel_res_true <= 1e-8
    assert pre.outer_iters <= 0.6 * plain.outer_iters
    assert sum(pre.inner_k) <= 0.5 * sum(plain.inner_k)


def test_colouring_makes_each_colour_independent():
    """The greedy colouring gives the 7-point stencil two colours (red-black: i + j + k even / odd); no two rows of a
    colour are coupled, so ILU(0) of the permuted matrix has diagonal colour blocks in L and U (each colour's rows of
    a triangular solve are independent), and it still solves the permuted system exactly up to the dropped fill."""
    A = workloads.convdiff(6, (20.0, 10.0, 5.0)).to_scipy().tocsr()
    n = A.shape[0]
    perm, colours, starts = ilu.colouring(A)
    assert len(starts) == 3 and sorted(perm.tolist()) == list(range(n))
    ijk = np.array([(i, j, k) for k in range(6) for j in range(6) for i in range(6)])
    parity = ijk.sum(axis=1) % 2
    assert np.array_equal(colours, parity) or np.array_equal(colours, 1 - parity)
    G = (A + A.T).tocoo()
    assert all(colours[r] != colours[c] for r, c in zip(G.row, G.col) if r != c)
    Pm = A[perm][:, perm].tocsr()
    L, U = ilu.ilu0(Pm)
    for c in range(2):
        a, e = starts[c], starts[c + 1]
        assert sp.tril(L[a:e, a:e], -1).nnz == 0 and sp.triu(U[a:e, a:e], 1).nnz == 0
    v = np.random.default_rng(3).standard_normal(n)
    z = ilu.ilu0_solve(L, U, v)
    np.testing.assert_allclose((L @ U) @ z, v, rtol=0, atol=1e-12 * np.abs(v).max())
    P = (L @ U).tocsr()
    pa = _pattern(Pm)
    Pd, Ad = P.toarray(), Pm.toarray()
    assert all(abs(Pd[i, j] - Ad[i, j]) <= 1e-12 * max(1.0, abs(Ad[i, j])) for i, j in pa)


def test_colouring_uses_the_pattern_not_the_values():
    """Two rows coupled by a skew-symmetric pair (a_01 = 1, a_10 = -1) are coupled in the pattern of A + A^T even
    though the values of A + A^T cancel there; they must get different colours, or the multicolour triangular solves
    would treat dependent rows as independent.  A stored zero is an edge too (it is part of ILU(0)'s pattern)."""
    A = sp.csr_matrix(np.array([[2.0, 1.0, 0.0, 0.0],
                                [-1.0, 2.0, 0.0, 0.0],
                                [0.0, 0.0, 2.0, 0.0],
                                [0.0, 0.0, 0.0, 2.0]]))
    _, colours, starts = ilu.colouring(A)
    assert colours[0] != colours[1] and len(starts) == 3
    Z = sp.csr_matrix((np.array([2.0, 0.0, 2.0, 2.0]), np.array([0, 2, 1, 2]), np.array([0, 2, 3, 4])), shape=(3, 3))
    _, cz, _ = ilu.colouring(Z)  # a_02 is a stored zero
    assert cz[0] != cz[2]
