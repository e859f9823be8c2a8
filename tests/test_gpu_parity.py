"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on identical seeded inputs.

Tolerances: the sketch pattern is integer work and must be bit-exact; FP64 first-cycle basis vectors agree to
1e-10 relative; both solvers reach ||b - A x|| / ||b|| <= 1e-8 with outer iteration counts within +-1.  Other
floating-point comparisons use tolerances derived in each test from the arithmetic involved.
"""
import numpy as np
import pytest

import workloads
from oracle import fgmres as ofg
from oracle import gmres as og
from oracle import sgmres as osg
from oracle import sketch as osk

from gpu_common import dev_vec, need_gpu, rel_err, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _solver(A, **opt):
    from paper_2506_18408_gb300 import Solver

    return Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=opt.pop("seed", 1), **opt)


# ---- sketch ------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,s,zeta,seed", [(4096, 120, 8, 1), (5003, 400, 8, 7), (1000, 8, 8, 3),
                                           (777, 50, 1, 11), (33333, 240, 16, 2**40 + 5)])
def test_sketch_pattern_bit_exact(n, s, zeta, seed):
    A = workloads.convdiff(n, (1.0,))  # any n x n matrix; only n matters here
    sv = _solver(A, seed=seed, zeta=zeta)
    rows, signs = sv.sketch_pattern(s)
    r_ref, s_ref = osk.sparse_sign_pattern(n, s, zeta, seed)
    assert np.array_equal(rows.cpu().numpy().astype(np.int64), r_ref)
    assert np.array_equal(signs.cpu().numpy(), s_ref)


@pytest.mark.parametrize("n,s,zeta", [(4096, 120, 8), (70001, 400, 8), (5000, 64, 1), (33333, 250, 16), (9000, 33, 3)])
def test_sketch_apply(n, s, zeta):
    A = workloads.convdiff(n, (1.0,))
    sv = _solver(A, seed=5, zeta=zeta)
    v = workloads.rhs(n, seed=9)
    c = sv.sketch(dev_vec(v), s).cpu().numpy()
    ref = osk.sketch_matrix(n, s, zeta, 5) @ v
    # each entry sums ~n*zeta/s terms of size |v|/sqrt(zeta): FP64 rounding bound well below 1e-13 relative
    assert rel_err(c, ref) <= 1e-13


def test_spmv_matches_scipy():
    for A in (workloads.convdiff(37, (20.0, 10.0)), workloads.random_zipf(20_011, seed=4)):
        sv = _solver(A)
        x = workloads.rhs(A.n, seed=2)
        y = sv.spmv(dev_vec(x)).cpu().numpy()
        assert rel_err(y, A.to_scipy() @ x) <= 1e-14


# ---- one inner cycle ---------------------------------------------------------------------------------------------
CYCLE_CASES = [
    ("cd2d_64", workloads.CONFIGS["cd2d_64"].build_matrix, 30, 120, 2),
    ("cd2d_37_t0", lambda: workloads.convdiff(37, (20.0, 10.0)), 25, 100, 0),
    ("zipf_20011_t4", lambda: workloads.random_zipf(20_011, seed=1), 40, 160, 4),
    ("cd3d_17_t1", lambda: workloads.convdiff(17, (50.0, 30.0, 10.0)), 30, 120, 1),
]


@pytest.mark.parametrize("name,make,m,s,t", CYCLE_CASES, ids=[c[0] for c in CYCLE_CASES])
def test_first_cycle_basis_fp64(name, make, m, s, t):
    A = make()
    b = workloads.rhs(A.n, seed=0)
    v = b / np.linalg.norm(b)
    sv = _solver(A)
    z, k, reason, B, y = sv.inner_cycle(dev_vec(v), m=m, s=s, k=t)
    S = osk.sketch_matrix(A.n, s, 8, 1)
    ref = osg.sgmres_cycle(A.to_scipy(), v, S, m, t, record=True)
    assert (k, reason) == (ref.k, ref.reason)
    B = B.cpu().numpy()
    for l in range(len(ref.basis)):
        assert rel_err(B[l], ref.basis[l]) <= 1e-10, (l, rel_err(B[l], ref.basis[l]))
    # z and y: the sketched LS amplifies rounding differences in S A B_k by up to cond(S A B_k) (about 1e12 for
    # the t = 0 power basis), so compare the inner residuals with a bound scaled by that condition number
    As = A.to_scipy()
    rg = np.linalg.norm(v - As @ z.cpu().numpy())
    ro = np.linalg.norm(v - As @ ref.z)
    kappa = np.linalg.cond(ref.sab)
    assert abs(rg - ro) <= 1e-6 * ro + 1e-15 * kappa, (rg, ro, kappa)


def test_identity_sketch_cycle_is_gmres():
    A = workloads.convdiff(7, (20.0, 10.0))  # n = 49
    b = workloads.rhs(A.n, seed=3)
    v = b / np.linalg.norm(b)
    sv = _solver(A, sketch_kind="identity")
    for t in (0, 2, 6):
        z, k, _, _, _ = sv.inner_cycle(dev_vec(v), m=6, s=A.n, k=t)
        x_ref = og.gmres_brute(A.to_scipy(), v, np.zeros(A.n), 6)
        assert k == 6
        assert rel_err(z.cpu().numpy(), x_ref) <= 1e-9


def test_c2_threshold_matches_oracle():
    A = workloads.convdiff(30, (50.0, 30.0))
    b = workloads.rhs(A.n, seed=0)
    v = b / np.linalg.norm(b)
    sv = _solver(A, cond_threshold=1e3)
    _, k, reason, _, _ = sv.inner_cycle(dev_vec(v), m=40, s=160, k=0)
    ref = osg.sgmres_cycle(A.to_scipy(), v, osk.sketch_matrix(A.n, 160, 8, 1), 40, 0, cond_thr=1e3)
    assert reason == osg.STOP_C2 and (k, reason) == (ref.k, ref.reason)


# ---- full solves -------------------------------------------------------------------------------------------------
def _compare_solve(A, b, m, s, t, tol=1e-8, max_outer=50, c3=True, x0=None, **opt):
    sv = _solver(A, max_outer=max_outer, c3=int(c3), **opt)
    x, info = sv.solve(dev_vec(b), None if x0 is None else dev_vec(x0), m=m, s=s, k=t, tol=tol)
    ref = ofg.fgmres(A.to_scipy(), b, x0, m=m, s=s, t=t, tol=tol, max_outer=max_outer, c3=c3)
    xh = x.cpu().numpy()
    rel = np.linalg.norm(b - A.to_scipy() @ xh) / np.linalg.norm(b)
    return info, ref, rel


SOLVE_CASES = [
    ("cd2d_64", workloads.CONFIGS["cd2d_64"].build_matrix, 30, 120, 2, 20, True),
    ("cd2d_64_noC3", workloads.CONFIGS["cd2d_64"].build_matrix, 30, 120, 2, 20, False),
    ("cd2d_64_t0", workloads.CONFIGS["cd2d_64"].build_matrix, 30, 120, 0, 20, True),
    ("zipf_20011", lambda: workloads.random_zipf(20_011, seed=0), 30, 120, 4, 50, True),
    ("cd3d_21_ragged", lambda: workloads.convdiff(21, (50.0, 30.0, 10.0)), 40, 160, 2, 50, True),
    # sketches larger than the single-CTA QR's 512 threads (several rows per thread) and not multiples of the 32-row
    # gather-list groups
    ("cd2d_48_s600", lambda: workloads.convdiff(48, (20.0, 10.0)), 30, 600, 2, 30, True),
    ("cd2d_48_s1000", lambda: workloads.convdiff(48, (20.0, 10.0)), 16, 1000, 2, 40, True),
]


@pytest.mark.parametrize("name,make,m,s,t,J,c3", SOLVE_CASES, ids=[c[0] for c in SOLVE_CASES])
def test_solve_parity_fp64(name, make, m, s, t, J, c3):
    A = make()
    b = workloads.rhs(A.n, seed=0, dist="uniform" if name.startswith("zipf") else "normal")
    info, ref, rel = _compare_solve(A, b, m, s, t, max_outer=J, c3=c3)
    assert info["status"] == 0 and ref.status == 0
    assert rel <= 1e-8 and ref.rel_res_true <= 1e-8
    assert abs(info["rel_res_true"] - rel) <= 1e-12 + 1e-6 * rel
    assert abs(info["outer_iters"] - ref.outer_iters) <= 1
    est = info["res_est"]
    assert all(b2 <= a2 * (1 + 1e-12) for a2, b2 in zip(est, est[1:])), est  # non-increasing (Algorithm 1)
    # the per-step estimates follow the oracle's while both run (different rounding, same iteration).  With t = 0
    # the power basis makes cond(S A B_k) ~1e13, so rounding differences of 1e-16 change each correction z_j by up
    # to ~1e-3 and the iterates drift apart; there only convergence and the iteration count are compared.
    if t > 0:
        for j in range(min(len(est), len(ref.est_hist)) - 1):
            assert abs(est[j] - ref.est_hist[j]) <= 1e-6 * ref.est_hist[j] + 1e-13, (j, est[j], ref.est_hist[j])
    # inner lengths agree except possibly where rule C3 compares two nearly equal numbers in the last cycle
    kk = info["inner_k"]
    common = min(len(kk), len(ref.inner_k)) - 1
    if t > 0:
        assert kk[:common] == ref.inner_k[:common]


def test_initial_guess_and_special_cases():
    from paper_2506_18408_gb300 import sfgmres as py

    A = workloads.convdiff(20, (20.0, 10.0))
    As = A.to_scipy()
    b = workloads.rhs(A.n, seed=1)
    sv = _solver(A, max_outer=20)
    # b = 0 -> x = 0
    x, info = sv.solve(dev_vec(np.zeros(A.n)), m=10, s=40, k=2)
    assert info["status"] == 0 and info["outer_iters"] == 0 and float(x.abs().max()) == 0.0
    # x0 exact -> returned unchanged, no iterations
    xs = np.linalg.solve(As.toarray(), b)
    x, info = sv.solve(dev_vec(b), dev_vec(xs), m=10, s=40, k=2)
    assert info["outer_iters"] == 0 and np.array_equal(x.cpu().numpy(), xs)
    # nonzero x0, aliased with x
    x0 = workloads.rhs(A.n, seed=2)
    xd = dev_vec(x0)
    x, info = sv.solve(dev_vec(b), xd, m=10, s=40, k=2, out=xd)
    ref = ofg.fgmres(As, b, x0, m=10, s=40, t=2, tol=1e-8, max_outer=20)
    assert info["status"] == 0 and abs(info["outer_iters"] - ref.outer_iters) <= 1
    assert np.linalg.norm(b - As @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(b)
    # NaN in b -> error, handle still usable
    bn = b.copy()
    bn[5] = np.nan
    with pytest.raises(py.SFGMRESError) as e:
        sv.solve(dev_vec(bn), m=10, s=40, k=2)
    assert e.value.code == py.ERR_NAN
    x, info = sv.solve(dev_vec(b), m=10, s=40, k=2)
    assert info["status"] == 0
    # invalid parameters
    for kw in (dict(m=0, s=40, k=2), dict(m=10, s=5, k=2), dict(m=10, s=40, k=9), dict(m=50, s=40, k=2)):
        with pytest.raises(py.SFGMRESError) as e:
            sv.solve(dev_vec(b), **kw)
        assert e.value.code == py.ERR_INVALID_ARG
    with pytest.raises(py.SFGMRESError):
        sv.solve(dev_vec(b), m=10, s=40, k=2, tol=0.0)


def test_budget_exhausted_returns_not_converged():
    A = workloads.convdiff(30, (50.0, 30.0))
    b = workloads.rhs(A.n, seed=0)
    sv = _solver(A, max_outer=2)
    x, info = sv.solve(dev_vec(b), m=5, s=40, k=2, tol=1e-12)
    ref = ofg.fgmres(A.to_scipy(), b, m=5, s=40, t=2, tol=1e-12, max_outer=2)
    assert info["status"] == 1 and info["outer_iters"] == 2 and ref.status == ofg.NOT_CONVERGED
    rel = np.linalg.norm(b - A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b)
    assert abs(rel - ref.rel_res_true) <= 1e-6 * ref.rel_res_true


def test_invalid_csr_rejected():
    from paper_2506_18408_gb300 import sfgmres as py

    A = workloads.convdiff(10, (1.0, 1.0))
    bad_col = A.col.copy()
    bad_col[7] = A.n + 3
    with pytest.raises(py.SFGMRESError):
        py.Solver(A.n, A.row_ptr, bad_col, A.val)
    bad_rp = A.row_ptr.copy()
    bad_rp[5], bad_rp[6] = bad_rp[6], bad_rp[5]
    with pytest.raises(py.SFGMRESError):
        py.Solver(A.n, bad_rp, A.col, A.val)


def test_host_buffers_give_the_same_result():
    A = workloads.convdiff(30, (20.0, 10.0))
    b = workloads.rhs(A.n, seed=0)
    sv = _solver(A, max_outer=20)
    xd, info_d = sv.solve(dev_vec(b), m=20, s=80, k=2)
    xh, info_h = sv.solve(b.copy(), m=20, s=80, k=2)
    assert isinstance(xh, np.ndarray)
    assert np.array_equal(xd.cpu().numpy(), xh)  # deterministic kernels: identical bits
    assert info_d["outer_iters"] == info_h["outer_iters"]


def test_repeat_solves_are_bitwise_reproducible():
    A = workloads.random_zipf(30_000, seed=3)
    b = workloads.rhs(A.n, seed=0, dist="uniform")
    sv = _solver(A)
    x1, _ = sv.solve(dev_vec(b), m=30, s=120, k=4)
    x2, _ = sv.solve(dev_vec(b), m=30, s=120, k=4)
    assert torch.equal(x1, x2)


def test_restarted_sgmres_follows_algorithm_2():
    """Restarted sGMRES (Algorithm 2: x_{c+1} = x_c + z_c, z_c one sGMRES cycle on r_c with rules C1 and C2) through
    the C ABI follows the oracle's cycle by cycle: the same residual history to 1e-6 relative (each cycle accepts all
    m = 30 columns here, far below the 1e15 condition threshold, so the two differ by rounding only) and the same
    iterate."""
    A = workloads.CONFIGS["cd2d_64"].build_matrix()
    b = workloads.rhs(A.n, seed=0)
    m, s, t, cycles = 30, 120, 2, 8
    sv = _solver(A)
    x, info = sv.solve_restarted(dev_vec(b), m=m, s=s, k=t, tol=1e-12, max_cycles=cycles)
    xr, hist, _ = ofg.restarted(A.to_scipy(), b, m=m, s=s, t=t, tol=1e-12, max_outer=cycles)
    assert info["status"] == 1 and info["cycles"] == cycles and len(hist) == cycles
    gh = info["rel_res_hist"]
    assert abs(gh[0] - 1.0) <= 1e-12  # x_0 = 0: r_0 = b
    for c in range(cycles):
        assert abs(gh[c + 1] - hist[c]) <= 1e-6 * hist[c] + 1e-15, (c, gh[c + 1], hist[c])
    xh = x.cpu().numpy()
    assert np.abs(xh - xr).max() <= 1e-6 * np.abs(xr).max()


def test_ffom_outer_variant_follows_the_oracle():
    """The FFOM outer variant (the iterate solves the square Hessenberg system; its residual is the one of Eq. 4)
    through the C ABI converges like the oracle's: outer iteration counts within 1, per-step FFOM residuals within
    1e-6 relative, true residual <= 1e-8.  The Arnoldi process is the FGMRES one, so an FGMRES solve on the same
    handle reports the same FFOM residuals (bit for bit) and least-squares estimates no larger than them."""
    A = workloads.CONFIGS["cd2d_64"].build_matrix()
    b = workloads.rhs(A.n, seed=0)
    m, s, t = 30, 120, 2
    sv = _solver(A, max_outer=30)
    sv.set("outer_variant", 1)
    x, info = sv.solve(dev_vec(b), m=m, s=s, k=t, tol=1e-8)
    ref = ofg.fgmres(A.to_scipy(), b, None, m=m, s=s, t=t, tol=1e-8, max_outer=30, variant="ffom")
    assert info["status"] == 0 and ref.status == 0
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - A.to_scipy() @ xh) / np.linalg.norm(b) <= 1e-8
    assert abs(info["outer_iters"] - ref.outer_iters) <= 1
    est = info["res_est"]
    assert est == info["ffom_res"]
    for j in range(min(len(est), len(ref.est_hist)) - 1):
        assert abs(est[j] - ref.est_hist[j]) <= 1e-6 * ref.est_hist[j] + 1e-13, (j, est[j], ref.est_hist[j])
    sv.set("outer_variant", 0)
    _, info0 = sv.solve(dev_vec(b), m=m, s=s, k=t, tol=1e-8)
    common = min(len(info0["ffom_res"]), len(est))
    assert info0["ffom_res"][:common] == info["ffom_res"][:common]
    assert all(a <= f for a, f in zip(info0["res_est"][:common], info["ffom_res"][:common]))


@pytest.mark.parametrize("name,make,m,s,t", [
    ("cd2d_64", workloads.CONFIGS["cd2d_64"].build_matrix, 30, 120, 2),
    ("zipf_20011", lambda: workloads.random_zipf(20_011, seed=0), 30, 120, 4),
], ids=["cd2d_64", "zipf_20011"])
def test_eq5_bound_traced_along_the_gpu_iteration(name, make, m, s, t):
    """Eq. 5 along the GPU's own iteration: ||r_j|| <= ||r~_{j-1}|| ||r_hat_j|| at every outer step j, with r_j the
    FGMRES residual (its Givens estimate), r~_{j-1} the FFOM residual of Eq. 4 of the previous step (beta at the first,
    Section 2.1) and r_hat_j = v_j - A z_j the true residual of inner cycle j, which the solver reports per step
    (inner_res) beside the sketched residual rho_k the cycle ended with (inner_rho, the estimate rule C3 uses).  Both
    per-step quantities follow the oracle's to 1e-6 relative while the two runs take the same steps."""
    A = make()
    b = workloads.rhs(A.n, seed=0, dist="uniform" if name.startswith("zipf") else "normal")
    sv = _solver(A, max_outer=50)
    _, info = sv.solve(dev_vec(b), m=m, s=s, k=t, tol=1e-8)
    ref = ofg.fgmres(A.to_scipy(), b, m=m, s=s, t=t, tol=1e-8, max_outer=50, trace=True)
    est, ffom, ir, rho = info["res_est"], info["ffom_res"], info["inner_res"], info["inner_rho"]
    J = info["outer_iters"]
    assert info["status"] == 0 and len(ir) == len(rho) == J
    prev = 1.0  # ||r~_0|| / ||b|| = beta / ||b|| = 1 with x0 = 0
    for j in range(J):
        assert 0.0 < ir[j] < 1.0 and 0.0 < rho[j] < np.inf
        assert est[j] <= prev * ir[j] * (1 + 1e-10) + 1e-15, (j, est[j], prev, ir[j])
        prev = ffom[j]
    for j in range(min(J, ref.outer_iters) - 1):
        assert abs(ir[j] - ref.rhat_hist[j]) <= 1e-6 * ref.rhat_hist[j], (j, ir[j], ref.rhat_hist[j])
        assert abs(rho[j] - ref.rho_hist[j]) <= 1e-6 * ref.rho_hist[j], (j, rho[j], ref.rho_hist[j])
