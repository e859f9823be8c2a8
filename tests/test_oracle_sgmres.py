"""Pins for the oracle's sketched-GMRES cycle (Eq. 3, Section 3: truncated Arnoldi, sketched LS, C1-C3)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import gmres as og
from oracle import sgmres as osg
from oracle import sketch as sk
from oracle.lowprec import round_bf16


def _problem(N=6, beta=(20.0, 10.0)):
    A = workloads.convdiff(N, beta).to_scipy()
    rng = np.random.default_rng(7)
    v = rng.standard_normal(A.shape[0])
    return A, v / np.linalg.norm(v)


@pytest.mark.parametrize("t", [0, 1, 2, 8])
def test_identity_sketch_reproduces_gmres(t):
    # With S = I the sketched LS is the GMRES LS over K_m(A, v), which does not depend on the basis (any t).
    A, v = _problem()
    n = A.shape[0]
    m = 7
    S = sk.sketch_matrix(n, n, kind="identity")
    cyc = osg.sgmres_cycle(A, v, S, m, t)
    assert cyc.k == m
    x_ref = og.gmres_brute(A, v, np.zeros(n), m)
    r_ref = np.linalg.norm(v - A @ x_ref)
    r = np.linalg.norm(v - A @ cyc.z)
    assert abs(r - r_ref) <= 1e-10 * max(r_ref, 1e-300) + 1e-13
    np.testing.assert_allclose(cyc.z, x_ref, rtol=0, atol=1e-9 * np.linalg.norm(x_ref))


def test_sketched_ls_matches_dense_lstsq():
    A, v = _problem(10)
    n = A.shape[0]
    S = sk.sketch_matrix(n, 60, 8, 3)
    cyc = osg.sgmres_cycle(A, v, S, 20, 2, record=True)
    k = cyc.k
    B = np.column_stack(cyc.basis[:k])
    SAB = S @ (A @ B)
    c0 = S @ v
    y_ref, *_ = np.linalg.lstsq(SAB, c0, rcond=None)
    np.testing.assert_allclose(cyc.y, y_ref, rtol=1e-9, atol=1e-12 * np.abs(y_ref).max())
    np.testing.assert_allclose(cyc.sab, SAB, rtol=0, atol=1e-13 * np.abs(SAB).max())
    # normal-equations optimality of the sketched residual
    res = c0 - SAB @ cyc.y
    assert np.linalg.norm(SAB.T @ res) <= 1e-10 * np.linalg.norm(SAB) * np.linalg.norm(c0)
    # rho_k is the sketched residual norm of the final LS
    assert abs(cyc.rho[-1] - np.linalg.norm(c0 - SAB @ y_ref)) <= 1e-10 * np.linalg.norm(c0)
    # z = B y
    np.testing.assert_allclose(cyc.z, B @ cyc.y, rtol=0, atol=1e-13 * np.abs(B @ cyc.y).max())


@pytest.mark.parametrize("t", [0, 1, 2, 4])
def test_truncated_arnoldi_properties(t):
    A, v = _problem(12, (50.0, 30.0))
    n = A.shape[0]
    S = sk.sketch_matrix(n, 80, 8, 3)
    m = 15
    cyc = osg.sgmres_cycle(A, v, S, m, t, record=True)
    B = np.column_stack(cyc.basis)
    np.testing.assert_allclose(np.linalg.norm(B, axis=0), 1.0, rtol=0, atol=1e-13)
    G = B.T @ B
    for i in range(B.shape[1]):
        for l in range(max(0, i - t), i):
            assert abs(G[i, l]) <= 1e-12, (i, l, G[i, l])
    # recurrence A b_i = sum_l h_l b_l + eta_i b_{i+1} over the window l = i-t+1..i
    for i, (h, eta) in enumerate(zip(cyc.h, cyc.eta)):
        lo = max(0, i - t + 1)
        recon = sum(hl * B[:, l] for hl, l in zip(h, range(lo, i + 1))) + eta * B[:, i + 1]
        np.testing.assert_allclose(recon, A @ B[:, i], rtol=0, atol=1e-12 * np.linalg.norm(A @ B[:, i]))
    if t == 0:
        # normalised power basis: b_{i+1} is A^i v scaled to unit norm
        p = v.copy()
        for i in range(B.shape[1]):
            np.testing.assert_allclose(B[:, i], p / np.linalg.norm(p), rtol=0, atol=1e-10)
            p = A @ p
    # span: the first k basis vectors span K_k(A, v) (small k, well conditioned)
    kk = 5
    K = np.empty((n, kk))
    K[:, 0] = v
    for i in range(1, kk):
        K[:, i] = A @ K[:, i - 1]
    coef, *_ = np.linalg.lstsq(B[:, :kk], K, rcond=None)
    assert np.linalg.norm(B[:, :kk] @ coef - K) <= 1e-9 * np.linalg.norm(K)


def test_full_arnoldi_when_t_at_least_m():
    A, v = _problem(8)
    n = A.shape[0]
    S = sk.sketch_matrix(n, 40, 8, 2)
    cyc = osg.sgmres_cycle(A, v, S, 10, 10, record=True)
    B = np.column_stack(cyc.basis)
    assert np.linalg.norm(B.T @ B - np.eye(B.shape[1])) <= 1e-12


def test_condition_proxy_and_c2():
    A, v = _problem(12, (50.0, 30.0))
    n = A.shape[0]
    S = sk.sketch_matrix(n, 100, 8, 4)
    cyc = osg.sgmres_cycle(A, v, S, 30, 0, record=True)  # power basis: ill-conditioned quickly
    conds = []
    for k in range(1, cyc.k + 1):
        SAB = cyc.sab[:, :k]
        c = np.linalg.cond(SAB)
        conds.append(c)
        assert cyc.kappa[k - 1] <= c * (1 + 1e-8)  # proxy is a lower bound of cond(R_k) = cond(SAB_k)
    assert all(b >= a * (1 - 1e-8) for a, b in zip(conds, conds[1:]))  # nested columns: cond non-decreasing
    # a low threshold makes C2 fire and drop the offending column
    thr = 1e2
    cyc2 = osg.sgmres_cycle(A, v, S, 30, 0, cond_thr=thr)
    assert cyc2.reason == osg.STOP_C2
    assert cyc2.kappa[cyc2.k] > thr and all(kp <= thr for kp in cyc2.kappa[: cyc2.k])
    assert len(cyc2.y) == cyc2.k


def test_c3_stops_at_first_step_meeting_the_bound():
    A, v = _problem(10)
    n = A.shape[0]
    S = sk.sketch_matrix(n, 80, 8, 3)
    full = osg.sgmres_cycle(A, v, S, 20, 2)
    scale = 3.0
    tol_abs = scale * full.rho[6] * 1.0000001
    cyc = osg.sgmres_cycle(A, v, S, 20, 2, bound_scale=scale, bound_tol=tol_abs)
    first = next(i for i, r in enumerate(full.rho) if scale * r <= tol_abs)
    assert cyc.reason == osg.STOP_C3 and cyc.k == first + 1
    assert cyc.k <= 7


def test_breakdown_on_invariant_subspace():
    # v is an eigenvector of a diagonal A: A v lies in span(v), so eta_1 = 0 and the cycle is exact with k = 1
    n = 50
    A = sp.diags(np.arange(1.0, n + 1)).tocsr()
    v = np.zeros(n)
    v[3] = 1.0
    S = sk.sketch_matrix(n, 20, 8, 1)
    cyc = osg.sgmres_cycle(A, v, S, 10, 2)
    assert cyc.k == 1 and cyc.reason == osg.STOP_BREAKDOWN
    np.testing.assert_allclose(A @ cyc.z, v, atol=1e-14)


def test_fp32_inner_close_to_fp64():
    A, v = _problem(16)
    n = A.shape[0]
    S = sk.sketch_matrix(n, 80, 8, 3)
    c64 = osg.sgmres_cycle(A, v, S, 15, 2, record=True)
    c32 = osg.sgmres_cycle(A, v, S, 15, 2, inner="fp32", record=True)
    assert c32.basis[3].dtype == np.float32
    for i in range(5):
        np.testing.assert_allclose(c32.basis[i], c64.basis[i], rtol=0, atol=5e-6)
    rr64 = np.linalg.norm(v - A @ c64.z)
    rr32 = np.linalg.norm(v - A @ c32.z)
    assert rr32 <= max(2 * rr64, 1e-5)


def test_round_bf16_against_enumeration():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(2000) * np.exp(rng.uniform(-20, 20, 2000))).astype(np.float32)
    x = np.concatenate([x, np.float32([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, -2.5, 0.0])])
    got = round_bf16(x)
    bits = x.view(np.uint32)
    lo = (bits & np.uint32(0xFFFF0000)).view(np.float32)
    hi = ((bits & np.uint32(0xFFFF0000)) + np.uint32(0x10000)).view(np.float32)
    dlo = np.abs(x.astype(np.float64) - lo)
    dhi = np.abs(hi.astype(np.float64) - x)
    even_lo = ((bits >> 16) & 1) == 0
    expect = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(even_lo, lo, hi)))
    assert np.array_equal(got.view(np.uint32), expect.view(np.uint32))
    assert got[-4] == np.float32(1.0) and got[-3] == np.float32(1.0 + 2**-6)
