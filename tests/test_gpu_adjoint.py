"""GPU: transpose solve, value updates, pattern gradient and the autograd Function (implicit differentiation)."""
import numpy as np
import pytest

import workloads
from oracle import fgmres as ofg

from gpu_common import dev_vec, need_gpu, rel_err, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _solver(A, **opt):
    from paper_2506_18408_gb300 import Solver

    return Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=1, **opt)


@pytest.mark.parametrize("make", [lambda: workloads.convdiff(32, (20.0, 10.0)),
                                  lambda: workloads.random_zipf(5003, seed=2)], ids=["cd2d_32", "zipf_5003"])
def test_transpose_solve_parity(make):
    A = make()
    At = A.to_scipy().T.tocsr()
    g = workloads.rhs(A.n, seed=6)
    sv = _solver(A, max_outer=40)
    lam, info = sv.solve(dev_vec(g), m=20, s=80, k=2, tol=1e-10, transpose=True)
    ref = ofg.fgmres(At, g, m=20, s=80, t=2, tol=1e-10, max_outer=40)
    rel = np.linalg.norm(g - At @ lam.cpu().numpy()) / np.linalg.norm(g)
    assert info["status"] == 0 and rel <= 1e-10
    assert abs(info["outer_iters"] - ref.outer_iters) <= 1


def test_pattern_outer_and_update_values():
    A = workloads.random_zipf(3001, seed=5)
    sv = _solver(A)
    u = workloads.rhs(A.n, seed=1)
    v = workloads.rhs(A.n, seed=2)
    out = torch.ones(A.nnz, dtype=torch.float64, device="cuda")
    sv.pattern_outer(dev_vec(u), dev_vec(v), -0.5, out)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    expect = 1.0 - 0.5 * u[rows] * v[A.col]
    assert rel_err(out.cpu().numpy(), expect) <= 1e-15
    # new values: the handle solves with them (forward and transpose) like a fresh handle
    vals2 = A.val * (1.0 + 0.1 * workloads.rhs(A.nnz, seed=3) ** 2)
    sv.update_values(dev_vec(vals2))
    fresh = workloads.CSR(A.n, A.row_ptr, A.col, vals2)
    sv2 = _solver(fresh)
    b = workloads.rhs(A.n, seed=9)
    for tr in (False, True):
        x1, _ = sv.solve(dev_vec(b), m=20, s=80, k=2, transpose=tr)
        x2, _ = sv2.solve(dev_vec(b), m=20, s=80, k=2, transpose=tr)
        assert torch.equal(x1, x2)


def test_autograd_matches_dense_adjoint():
    from paper_2506_18408_gb300 import sfgmres_solve_autograd

    A = workloads.convdiff(8, (50.0, 30.0, 10.0))  # n = 512
    sv = _solver(A)
    nrhs = 3
    B = workloads.rhs(A.n, seed=0, nrhs=nrhs)
    Xs = workloads.rhs(A.n, seed=0, stream=workloads.STREAM_XSTAR, nrhs=nrhs)
    vals = torch.tensor(A.val, dtype=torch.float64, device="cuda", requires_grad=True)
    b = torch.tensor(B, dtype=torch.float64, device="cuda", requires_grad=True)
    x = sfgmres_solve_autograd(sv, vals, b, m=30, s=120, k=2, tol=1e-13)
    loss = ((x - torch.tensor(Xs, device="cuda")) ** 2).sum()
    loss.backward()
    Ad = A.to_scipy().toarray()
    X = np.linalg.solve(Ad, B.T).T
    Lam = np.linalg.solve(Ad.T, 2 * (X - Xs).T).T
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    gA = -(Lam[:, rows] * X[:, A.col]).sum(axis=0)
    assert rel_err(x.detach().cpu().numpy(), X) <= 1e-11
    assert rel_err(b.grad.cpu().numpy(), Lam) <= 1e-10
    assert rel_err(vals.grad.cpu().numpy(), gA) <= 1e-10


def _fd_check(N, nrhs, nent, m, s, seed=2):
    """Central differences (h = 1e-6) of L = sum ||x - x*||^2 against the adjoint gradient, forward solves at
    tol 1e-13.  FD error: truncation O(h^2) (zero in b, where L is quadratic) plus the rounding of the two values of
    L, up to about 4 eps |L| / (2h); a solve error that is smooth in the data contributes O(tol).  The bound used is
    1e-5 |g| + 2 eps |L| / h."""
    from paper_2506_18408_gb300 import sfgmres_solve_autograd

    A = workloads.convdiff(N, (50.0, 30.0, 10.0))
    sv = _solver(A, max_outer=60)
    B = workloads.rhs(A.n, seed=0, nrhs=nrhs)
    Xs = torch.tensor(workloads.rhs(A.n, seed=0, stream=workloads.STREAM_XSTAR, nrhs=nrhs), device="cuda")
    vals = torch.tensor(A.val, dtype=torch.float64, device="cuda", requires_grad=True)
    b = torch.tensor(B, dtype=torch.float64, device="cuda", requires_grad=True)
    tol = 1e-13

    def L(vv, bb):
        with torch.no_grad():
            x = sfgmres_solve_autograd(sv, vv, bb, m=m, s=s, k=2, tol=tol)
            return float(((x - Xs) ** 2).sum())

    x = sfgmres_solve_autograd(sv, vals, b, m=m, s=s, k=2, tol=tol)
    Lval = ((x - Xs) ** 2).sum()
    Lval.backward()
    eps = np.finfo(np.float64).eps
    gv, gb = vals.grad.clone(), b.grad.clone()
    rng = np.random.default_rng([seed, workloads.STREAM_SAMPLE])
    h = 1e-6
    fd_noise = 2 * eps * abs(float(Lval.detach())) / h
    v0 = vals.detach().clone()
    b0 = b.detach().clone()
    for p in rng.choice(A.nnz, nent // 2, replace=False):
        vp, vm = v0.clone(), v0.clone()
        vp[p] += h
        vm[p] -= h
        fd = (L(vp, b0) - L(vm, b0)) / (2 * h)
        assert abs(fd - float(gv[p])) <= 1e-5 * abs(float(gv[p])) + fd_noise, (p, fd, float(gv[p]), fd_noise)
    for flat in rng.choice(nrhs * A.n, nent - nent // 2, replace=False):
        r, i = divmod(int(flat), A.n)
        bp, bm = b0.clone(), b0.clone()
        bp[r, i] += h
        bm[r, i] -= h
        fd = (L(v0, bp) - L(v0, bm)) / (2 * h)
        assert abs(fd - float(gb[r, i])) <= 1e-5 * abs(float(gb[r, i])) + fd_noise, (r, i, fd, float(gb[r, i]))


def test_finite_differences_small():
    _fd_check(16, 4, 16, 30, 120)


def test_finite_differences_3d_64_16rhs():
    # the differentiation workload: 3D convection-diffusion 64^3, 16 right-hand sides, 32 random entries
    # (half in b, half in the values of A), m = 50, k = 2, s = 200
    _fd_check(64, 16, 32, 50, 200)
