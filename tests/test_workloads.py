"""Checks of the seeded problem generators against closed forms."""
import numpy as np
import scipy.sparse as sp

import workloads


def test_nnz_counts():
    assert workloads.convdiff(64, (20.0, 10.0)).nnz == 20_224
    assert workloads.convdiff(64, (50.0, 30.0, 10.0)).nnz == 1_810_432


def test_laplacian_special_case_eigenvalues():
    # beta = 0: h^2-scaled 5-point Laplacian with eigenvalues 4 - 2cos(i pi h) - 2cos(j pi h)
    N = 9
    A = workloads.convdiff(N, (0.0, 0.0)).to_scipy().toarray()
    h = 1.0 / (N + 1)
    k = np.arange(1, N + 1)
    lam1 = 2 - 2 * np.cos(k * np.pi * h)
    expect = np.sort((lam1[:, None] + lam1[None, :]).ravel())
    got = np.sort(np.linalg.eigvalsh(A))
    np.testing.assert_allclose(got, expect, atol=1e-12)
    # 1D/3D consistency: 3D Laplacian is the Kronecker sum of three 1D ones
    A1 = workloads.convdiff(N, (0.0,)).to_scipy()
    I = sp.identity(N)
    A3 = sp.kron(sp.kron(I, I), A1) + sp.kron(sp.kron(I, A1), I) + sp.kron(sp.kron(A1, I), I)
    B3 = workloads.convdiff(N, (0.0, 0.0, 0.0)).to_scipy()
    assert abs(A3 - B3).max() < 1e-15


def test_upwind_row():
    N, beta = 8, (20.0, -10.0)
    A = workloads.convdiff(N, beta).to_scipy().toarray()
    h = 1.0 / (N + 1)
    i = 3 + 4 * N  # interior point x=3, y=4
    assert np.isclose(A[i, i], 4 + h * 30)
    assert np.isclose(A[i, i - 1], -1 - 20 * h) and np.isclose(A[i, i + 1], -1)  # beta_x > 0: upwind is -x
    assert np.isclose(A[i, i + N], -1 - 10 * h) and np.isclose(A[i, i - N], -1)  # beta_y < 0: upwind is +y
    # discrete operator applied to a linear function reproduces beta . grad u (times h^2) in the interior
    xs = (np.arange(N) + 1) * h
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    u = (2 * X + 3 * Y).ravel()
    interior = np.zeros((N, N), dtype=bool)
    interior[1:-1, 1:-1] = True
    lhs = (A @ u)[interior.ravel()]
    np.testing.assert_allclose(lhs, h * h * (20 * 2 + (-10) * 3), atol=1e-12)


def test_zipf_matrix_structure():
    Z = workloads.random_zipf(20_000, seed=2)
    L = np.diff(Z.row_ptr)
    assert L.min() >= 4 and L.max() <= 256
    rows = np.repeat(np.arange(Z.n), L)
    same = rows[1:] == rows[:-1]
    assert np.all(np.diff(Z.col.astype(np.int64))[same] > 0)  # sorted, distinct
    A = Z.to_scipy()
    d = A.diagonal()
    off = np.asarray(abs(A).sum(axis=1)).ravel() - np.abs(d)
    np.testing.assert_allclose(d, 1.2 * off, rtol=1e-12)
    assert 15 < Z.nnz / Z.n < 35


def test_rhs_streams_independent():
    a = workloads.rhs(100, seed=0)
    b = workloads.rhs(100, seed=0, stream=workloads.STREAM_XSTAR)
    assert not np.allclose(a, b)
    u = workloads.rhs(1000, seed=0, dist="uniform")
    assert u.min() >= -1 and u.max() <= 1
