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


def test_block_diag_round_trip_and_problem_slices():
    mats = [workloads.convdiff(5, (1.0, 2.0)), workloads.random_zipf(40, seed=1), workloads.convdiff(3, (0.0,))]
    A = workloads.block_diag(mats)
    assert A.n == sum(M.n for M in mats) and A.nnz == sum(M.nnz for M in mats)
    assert list(A.sys_n) == [M.n for M in mats]
    D = A.to_scipy().toarray()
    off = 0
    for M in mats:
        blk = D[off:off + M.n, off:off + M.n]
        np.testing.assert_array_equal(blk, M.to_scipy().toarray())
        D[off:off + M.n, off:off + M.n] = 0.0
        off += M.n
    assert not D.any()  # nothing outside the diagonal blocks
    for M, B in zip(mats, workloads.split_blocks(A)):
        np.testing.assert_array_equal(B.row_ptr, M.row_ptr)
        np.testing.assert_array_equal(B.col, M.col)
        np.testing.assert_array_equal(B.val, M.val)
    sl = workloads.problem_slices(A.sys_n, 3)
    assert [q for q, _, _ in sl] == [0, 0, 0, 1, 1, 1, 2, 2, 2]
    starts = [a for _, a, _ in sl]
    lens = [n for _, _, n in sl]
    assert starts[0] == 0 and all(a + n == a2 for a, n, a2 in zip(starts, lens, starts[1:]))
    assert starts[-1] + lens[-1] == 3 * A.n


def test_convdiff_batch_recipe():
    A = workloads.convdiff_batch(40, 32, 512, 50.0, seed=0)
    N = np.sqrt(A.sys_n).round().astype(np.int64)
    assert np.all(N * N == A.sys_n) and N.min() >= 32 and N.max() <= 512
    # 5-point stencil: nnz = 5 N^2 - 4 N per system
    assert A.nnz == int(np.sum(5 * N * N - 4 * N))
    b = workloads.batch_rhs(A.sys_n, 4, seed=0)
    assert b.shape == (4 * A.n,)
    cfg = workloads.CONFIGS["batch_512"]
    assert (cfg.nrhs, cfg.m, cfg.t, cfg.s, cfg.precision) == (4, 40, 2, 160, "fp32")


def test_roofline_byte_counts_match_the_per_step_figures():
    """bench.py's algorithmic bytes per inner step (A once with column indices and row pointers; b_i read, w written
    and read back, the t window vectors for the update and t - 1 of them again for the dots, b_{i+1} written; the
    sketch hashed, so no bytes for S) give, for the 3D convection-diffusion 128^3 workload with t = 2, about 301 MB
    per FP64 step and 184 MB per FP32 step; the fused inner kernel's own count (gather lists and block partials
    instead of the update's vectors) is 268.6 MB in FP64."""
    import bench

    cfg = workloads.CONFIGS["cd3d_128"]
    n, nnz = 128 ** 3, 14_581_760
    assert cfg.t == 2
    fp64 = bench.alg_bytes_inner_step(n, nnz, cfg.t, 8)
    fp32 = bench.alg_bytes_inner_step(n, nnz, cfg.t, 4)
    assert fp64 == nnz * 12 + 4 * (n + 1) + 7 * n * 8
    assert abs(fp64 / 1e6 - 300.8) < 0.1 and abs(fp32 / 1e6 - 183.8) < 0.1
    nblk = -(-n // 7296)
    assert nblk == 288
    k1 = bench.alg_bytes_inner_spmv(n, nnz, cfg.t, cfg.zeta, cfg.s, nblk, 8)
    assert abs(k1 / 1e6 - 268.6) < 0.1


def test_whole_solve_byte_count():
    """bench.py's bytes of a whole solve of one problem (the batch roofline): its inner steps at the per-step count
    (FP32 values and basis for FP32 inner cycles), z = B y once per cycle, and the outer steps; written out for a
    problem of 2 outer steps and 10 inner steps."""
    import bench

    n, nnz, t = 1000, 4960, 2
    step = nnz * (4 + 4) + 4 * (n + 1) + (2 * t + 3) * n * 4
    gemv = (10 + 2) * n * 4 + 2 * 8 * n
    outer = sum(nnz * 12 + 4 * (n + 1) + 16 * n + (4 * j + 3) * n * 8 for j in range(2))
    assert bench.alg_bytes_solve(n, nnz, t, 4, 4, 10, 2) == 10 * step + gemv + outer
    assert bench.alg_bytes_inner_step_prec(n, nnz, t, 8, 8) == bench.alg_bytes_inner_step(n, nnz, t, 8)
