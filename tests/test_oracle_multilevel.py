"""Pins of the oracle's multi-level FGMRES (Section 5: the outer FGMRES capped at a small basis and used as the
preconditioner of a higher-level FGMRES, recursively; the lowest level preconditioned by an sGMRES cycle).

* A child of budget one step is one sGMRES cycle followed by the optimal scaling of its correction; FGMRES's iterate
  depends only on span{z_1..z_j}, so the two-level method reproduces plain FGMRES-sGMRES step for step (C3 off, and
  C3 on, where the child's rule C3 -- its FFOM residual 1 times rho against tol ||b|| / ||r~_{j-1}|| -- is
  algebraically the parent's).
* With rule C3 on the child of the first step is asked for tol ||b|| / beta, and Eq. 5 gives ||r_1|| <= beta
  ||r_hat_1||: a child with budget enough to get there makes the top level converge in one step.
* Two and three levels converge to 1e-8 on the 2D workload with non-increasing top-level residuals (Algorithm 1) and
  the Eq. 5 bound at every top-level step, with the true residual of each child.
"""
import numpy as np
import pytest

import workloads
from oracle import fgmres as ofg

pytestmark = pytest.mark.filterwarnings("ignore")


def _cd2d():
    cfg = workloads.CONFIGS["cd2d_64"]
    A = cfg.build_matrix().to_scipy()
    return A, cfg.build_rhs(A.shape[0])


@pytest.mark.parametrize("c3", [False, True])
def test_budget_one_child_reproduces_plain_fgmres(c3):
    A, b = _cd2d()
    kw = dict(m=30, s=120, t=2, tol=1e-8, max_outer=20, c3=c3)
    plain = ofg.fgmres(A, b, **kw)
    two = ofg.fgmres(A, b, level_steps=(1,), **kw)
    assert two.status == plain.status == ofg.CONVERGED
    assert two.outer_iters == plain.outer_iters
    assert all(k == 1 for k in two.inner_k)
    for e2, e1 in zip(two.est_hist, plain.est_hist):
        assert abs(e2 - e1) <= 1e-9 * e1, (e2, e1)
    assert abs(two.rel_res_true - plain.rel_res_true) <= 1e-6 * plain.rel_res_true


def test_child_to_the_eq5_tolerance_converges_in_one_top_step():
    A, b = _cd2d()
    r = ofg.fgmres(A, b, m=30, s=120, t=2, tol=1e-8, max_outer=5, c3=True, level_steps=(40,), trace=True)
    assert r.status == ofg.CONVERGED and r.outer_iters == 1 and r.rel_res_true <= 1e-8
    assert r.inner_reason == [3]  # the child met tol ||b|| / beta
    assert r.rhat_hist[0] <= 1e-8 * (1 + 1e-6)  # beta = ||b|| with x0 = 0


@pytest.mark.parametrize("levels", [(3,), (4, 2)], ids=["two_levels", "three_levels"])
def test_multilevel_converges_with_the_eq5_bound(levels):
    A, b = _cd2d()
    r = ofg.fgmres(A, b, m=20, s=80, t=2, tol=1e-8, max_outer=30, c3=True, level_steps=levels, trace=True)
    assert r.status == ofg.CONVERGED and r.rel_res_true <= 1e-8
    assert all(k <= levels[0] for k in r.inner_k)
    est = r.est_hist
    assert all(b2 <= a2 * (1 + 1e-12) for a2, b2 in zip(est, est[1:]))
    prev = 1.0  # ||r~_{-1}|| / ||b|| = beta / ||b||
    for j in range(r.outer_iters):
        assert est[j] <= prev * r.rhat_hist[j] * (1 + 1e-10) + 1e-15, (j, est[j], prev, r.rhat_hist[j])
        prev = r.ffom_hist[j]
