"""Pins for the oracle's FGMRES/FFOM (Algorithm 1, Eq. 4, Eq. 5) and Algorithm 2."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import fgmres as ofg
from oracle import gmres as og


def _cd(N=12, beta=(50.0, 30.0)):
    A = workloads.convdiff(N, beta).to_scipy()
    b = workloads.rhs(A.shape[0], seed=3)
    return A, b


def test_exact_preconditioner_converges_in_one_step():
    # Section 2.1: rhat_1 = 0 gives the exact iterate after one outer step
    A, b = _cd(5)
    Ad = A.toarray()
    res = ofg.fgmres(A, b, m=1, s=1, t=0, tol=1e-13, precond=lambda v: np.linalg.solve(Ad, v))
    assert res.outer_iters == 1 and res.rel_res_true <= 1e-12


def test_identity_sketch_full_inner_space_is_exact():
    # S = I and m = n: the inner sGMRES is full GMRES on K_n, i.e. an exact solve (small well-conditioned n)
    A, b = _cd(4)  # n = 16
    n = A.shape[0]
    res = ofg.fgmres(A, b, m=n, s=n, t=n, tol=1e-12, sketch_kind="identity", c3=False)
    assert res.outer_iters == 1 and res.rel_res_true <= 1e-11


@pytest.mark.parametrize("t,orth", [(2, "mgs"), (0, "mgs"), (2, "cgs2")])
def test_identities_along_the_iteration(t, orth):
    A, b = _cd(12)
    n = A.shape[0]
    res = ofg.fgmres(A, b, m=8, s=40, t=t, tol=1e-10, max_outer=25, c3=False, outer_orth=orth,
                     record=True, track_true=True)
    assert res.status == ofg.CONVERGED
    V, Z, H = res.V, res.Z, res.H
    J = Z.shape[1]
    nb = np.linalg.norm(b)
    # Arnoldi-like relation A Z_J = V_{J+1} H_J
    AZ = A @ Z
    assert np.linalg.norm(AZ - V @ H) <= 1e-12 * np.linalg.norm(AZ)
    # CGS2 keeps V orthonormal to working precision; MGS loses orthogonality as the residual falls (but stays
    # backward stable), so only a loose check applies there
    assert np.linalg.norm(V.T @ V - np.eye(J + 1)) <= (1e-13 if orth == "cgs2" else 1e-3)
    for j in range(1, J + 1):
        # FGMRES iterate = brute-force minimiser over x0 + span(Z_j)
        y = np.linalg.lstsq(AZ[:, :j], b, rcond=None)[0]
        r_brute = np.linalg.norm(b - AZ[:, :j] @ y) / nb
        assert abs(res.est_hist[j - 1] - r_brute) <= 1e-9 * r_brute + 1e-14
        assert abs(res.true_hist[j - 1] - r_brute) <= 1e-7 * r_brute + 1e-13
        # FFOM residual of Eq. 4 vs the explicit FFOM iterate
        yF = np.linalg.solve(H[:j, :j], np.eye(j)[:, 0] * res.beta)
        rF = np.linalg.norm(b - A @ (Z[:, :j] @ yF)) / nb
        assert abs(res.ffom_hist[j - 1] - rF) <= 1e-6 * rF + 1e-13
        # ||r_j|| <= ||rtilde_j||
        assert res.est_hist[j - 1] <= res.ffom_hist[j - 1] * (1 + 1e-10)
        # Eq. 5 bound ||r_j|| <= ||rtilde_{j-1}|| ||rhat_j||, first step ||r_1|| <= beta ||rhat_1||
        prev = res.beta / nb if j == 1 else res.ffom_hist[j - 2]
        assert res.est_hist[j - 1] <= prev * res.rhat_hist[j - 1] * (1 + 1e-10) + 1e-15
    # non-increasing residual norms
    assert all(b2 <= a2 * (1 + 1e-12) for a2, b2 in zip(res.est_hist, res.est_hist[1:]))
    assert all(b2 <= a2 * (1 + 1e-9) for a2, b2 in zip(res.true_hist, res.true_hist[1:]))


def test_ffom_variant_residual_matches_eq4():
    A, b = _cd(10)
    res = ofg.fgmres(A, b, m=8, s=40, t=2, tol=1e-9, max_outer=30, c3=False, variant="ffom", record=True,
                     track_true=True)
    for j in range(len(res.est_hist)):
        assert abs(res.est_hist[j] - res.true_hist[j]) <= 1e-6 * res.true_hist[j] + 1e-13


def test_restarted_residual_equals_inner_residual():
    # Algorithm 2: r_j = rhat_j
    A, b = _cd(10)
    _, hist, rhat = ofg.restarted(A, b, m=8, s=40, t=2, tol=1e-9, max_outer=10)
    nb = np.linalg.norm(b)
    # equal up to rounding of the two evaluations (b - A x_j versus r_{j-1} - A z_j)
    np.testing.assert_allclose(np.array(hist) * nb, rhat, rtol=1e-8, atol=1e-14 * nb)


def test_config1_converges_nonincreasing_and_t0():
    cfg = workloads.CONFIGS["cd2d_64"]
    A = cfg.build_matrix().to_scipy()
    b = cfg.build_rhs(A.shape[0])
    for t in (cfg.t, 0):  # t = 0 (power basis) still converges under FGMRES (Section 4.1)
        res = ofg.fgmres(A, b, m=cfg.m, s=cfg.s, t=t, tol=cfg.tol, max_outer=cfg.max_outer, track_true=True)
        assert res.status == ofg.CONVERGED and res.rel_res_true <= cfg.tol
        assert all(y <= x * (1 + 1e-12) for x, y in zip(res.est_hist, res.est_hist[1:]))


def test_special_cases():
    A, b = _cd(6)
    n = A.shape[0]
    res = ofg.fgmres(A, np.zeros(n), m=5, s=20, t=2)
    assert res.outer_iters == 0 and np.all(res.x == 0)
    xs = np.linalg.solve(A.toarray(), b)
    res = ofg.fgmres(A, b, xs, m=5, s=20, t=2, tol=1e-8)
    assert res.outer_iters == 0 and np.array_equal(res.x, xs)


def test_fig2_setting_superlinear_vs_restarted():
    # Section 2.3: diag(1..1000), GMRES(5) as preconditioner: FGMRES accelerates, GMRES(5) converges linearly
    n = 1000
    A = sp.diags(np.arange(1.0, n + 1)).tocsr()
    b = workloads.rhs(n, seed=5)
    res = ofg.fgmres(A, b, m=5, s=n, t=5, tol=1e-8, max_outer=80, sketch_kind="identity", c3=False)
    _, hist = og.gmres_restarted(A, b, np.zeros(n), 5, 80)
    assert res.status == ofg.CONVERGED
    reached = next((i for i, h in enumerate(hist) if h <= 1e-8), None)
    assert reached is None or reached > 1.5 * res.outer_iters
    e = np.array(res.est_hist)
    early = (e[10] / e[0]) ** (1 / 10)
    late = (e[-1] / e[-11]) ** (1 / 10)
    assert late < early  # the per-step reduction factor improves (superlinear)


@pytest.mark.slow
def test_fig1_setting_restarted_stagnates_fgmres_converges():
    # Section 2.1: A = randn(1000) + 30 I, inner GMRES(100); restarted GMRES(100) stagnates
    n = 1000
    rng = np.random.default_rng(0)
    Ad = rng.standard_normal((n, n)) + 30.0 * np.eye(n)
    A = sp.csr_matrix(Ad)
    b = rng.standard_normal(n)
    _, hist = og.gmres_restarted(A, b, np.zeros(n), 100, 15)
    res = ofg.fgmres(A, b, m=100, s=n, t=100, tol=1e-8, max_outer=40, sketch_kind="identity", c3=False)
    assert res.status == ofg.CONVERGED
    assert hist[-1] > 1e-3


def test_truncation_sweep_lengthens_c2_driven_cycles():
    """Section 4's observation on the truncation parameter t, with a large k_max and rule C2 alone deciding the
    cycle length (C3 off): larger t gives better-conditioned bases and so longer cycles; t = 0 (a power basis, no
    orthogonalisation) ends every cycle by C2 well before k_max, yet FGMRES still converges; from t = 2 on this 2D
    convection-diffusion matrix the first cycle reaches k_max (C1)."""
    A = workloads.convdiff(32, (20.0, 10.0)).to_scipy().tocsr()
    b = workloads.rhs(A.shape[0], seed=0)
    m = 300
    first = []
    for t in range(6):
        r = ofg.fgmres(A, b, None, m=m, s=600, t=t, tol=1e-8, max_outer=40, c3=False)
        assert r.status == 0 and r.rel_res_true <= 1e-8, t
        first.append(r.inner_k[0])
        if t == 0:
            assert all(k < m for k in r.inner_k) and set(r.inner_reason) == {2} and r.outer_iters > 3
        if t >= 2:
            assert r.inner_k[0] == m and r.inner_reason[0] == 1
    assert all(a <= b2 for a, b2 in zip(first, first[1:])), first
