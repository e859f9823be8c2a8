"""Pins for the adjoint (implicit differentiation of x = A^{-1} b) on the oracle side."""
import numpy as np
import scipy.sparse as sp

import workloads
from oracle import fgmres as ofg


def test_transpose_solve_is_adjoint():
    A = workloads.convdiff(12, (50.0, 30.0)).to_scipy()
    g = workloads.rhs(A.shape[0], seed=4)
    res = ofg.fgmres(A.T.tocsr(), g, m=10, s=40, t=2, tol=1e-12, max_outer=40)
    lam_ref = np.linalg.solve(A.toarray().T, g)
    assert res.status == ofg.CONVERGED
    np.testing.assert_allclose(res.x, lam_ref, rtol=0, atol=1e-9 * np.abs(lam_ref).max())


def test_gradient_formula_against_finite_differences():
    # L = ||A^{-1} b - x*||^2: dL/db = A^{-T} g, dL/dA_ij = -(A^{-T} g)_i x_j on the pattern, g = 2 (x - x*)
    A = workloads.convdiff(4, (20.0, 10.0, 5.0)).to_scipy().tocsr()  # n = 64
    n = A.shape[0]
    b = workloads.rhs(n, seed=1)
    xs = workloads.rhs(n, seed=2)

    def loss(vals, bb):
        M = sp.csr_matrix((vals, A.indices, A.indptr), shape=A.shape).toarray()
        x = np.linalg.solve(M, bb)
        return float(np.sum((x - xs) ** 2)), x

    L0, x = loss(A.data, b)
    lam = np.linalg.solve(A.toarray().T, 2 * (x - xs))
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    gA = -lam[rows] * x[A.indices]
    h = 1e-6
    for p in (0, 5, 17, 100, A.nnz - 1):
        vp = A.data.copy(); vp[p] += h
        vm = A.data.copy(); vm[p] -= h
        fd = (loss(vp, b)[0] - loss(vm, b)[0]) / (2 * h)
        assert abs(fd - gA[p]) <= 1e-6 * max(1.0, abs(gA[p]))
    for i in (0, 31, 63):
        bp = b.copy(); bp[i] += h
        bm = b.copy(); bm[i] -= h
        fd = (loss(A.data, bp)[0] - loss(A.data, bm)[0]) / (2 * h)
        assert abs(fd - lam[i]) <= 1e-6 * max(1.0, abs(lam[i]))
