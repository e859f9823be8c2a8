"""GPU parity of the multi-level FGMRES (Section 5's outlook: an FGMRES with a capped basis used as the preconditioner
of a higher-level FGMRES, recursively; sGMRES cycles at the lowest level) through sfgmres_solve_multilevel, against
the oracle's ``fgmres(..., level_steps=...)`` on the same seeded inputs.

* A lower level with a budget of one step is one sGMRES cycle whose correction is optimally rescaled, which leaves
  FGMRES's iterates unchanged: the two-level solve reproduces the plain solve of the same handle step for step
  (residual estimates within 1e-9 relative, the same outer count), with rule C3 off and on.
* Two and three levels against the oracle: both reach 1e-8 (recomputed), top-level outer counts within 1, the steps
  each lower level took for a top-level step equal for every step but the last (rule C3 compares two nearly equal
  numbers there), top-level residual estimates within 1e-6 relative while both run, and the bound of Eq. 5 along
  the GPU's iteration with the true residual ||v_j - A z_j|| of each lower-level run.
* With C3 on, a lower level given budget enough reaches the tolerance Eq. 5 asks for, and the top level converges in
  one step.
"""
import numpy as np
import pytest

import workloads
from oracle import fgmres as ofg

from gpu_common import dev_vec, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def cd2d():
    cfg = workloads.CONFIGS["cd2d_64"]
    A = cfg.build_matrix()
    return A, cfg.build_rhs(A.n)


def _solver(A, **opt):
    from paper_2506_18408_gb300 import Solver

    return Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=1, **opt)


@pytest.mark.parametrize("c3", [0, 1])
def test_budget_one_level_reproduces_plain_solve(cd2d, c3):
    A, b = cd2d
    sv = _solver(A, max_outer=20, c3=c3)
    _, plain = sv.solve(dev_vec(b), m=30, s=120, k=2, tol=1e-8)
    x, two = sv.solve(dev_vec(b), m=30, s=120, k=2, tol=1e-8, level_steps=[1])
    assert plain["status"] == two["status"] == 0
    assert two["outer_iters"] == plain["outer_iters"] and all(k == 1 for k in two["inner_k"])
    for e2, e1 in zip(two["res_est"], plain["res_est"]):
        assert abs(e2 - e1) <= 1e-9 * e1, (e2, e1)
    rel = np.linalg.norm(b - A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b)
    assert rel <= 1e-8


@pytest.mark.parametrize("levels", [(3,), (4, 2)], ids=["two_levels", "three_levels"])
def test_multilevel_against_oracle(cd2d, levels):
    A, b = cd2d
    As = A.to_scipy()
    sv = _solver(A, max_outer=30)
    x, info = sv.solve(dev_vec(b), m=20, s=80, k=2, tol=1e-8, level_steps=list(levels))
    ref = ofg.fgmres(As, b, m=20, s=80, t=2, tol=1e-8, max_outer=30, c3=True, level_steps=levels, trace=True)
    rel = float(np.linalg.norm(b - As @ x.cpu().numpy()) / np.linalg.norm(b))
    print(f"{levels}: GPU outer {info['outer_iters']} child steps {info['inner_k']} sGMRES steps "
          f"{info['total_inner']} | oracle outer {ref.outer_iters} child steps {ref.inner_k}")
    assert info["status"] == 0 and ref.status == ofg.CONVERGED
    assert rel <= 1e-8 and ref.rel_res_true <= 1e-8
    assert abs(rel - info["rel_res_true"]) <= 1e-12 + 1e-6 * rel
    assert abs(info["outer_iters"] - ref.outer_iters) <= 1
    common = min(len(info["inner_k"]), len(ref.inner_k)) - 1
    assert info["inner_k"][:common] == ref.inner_k[:common]
    est, ffom, ir = info["res_est"], info["ffom_res"], info["inner_res"]
    for j in range(min(len(est), len(ref.est_hist)) - 1):
        assert abs(est[j] - ref.est_hist[j]) <= 1e-6 * ref.est_hist[j], (j, est[j], ref.est_hist[j])
        assert abs(ir[j] - ref.rhat_hist[j]) <= 1e-6 * ref.rhat_hist[j], (j, ir[j], ref.rhat_hist[j])
    assert all(b2 <= a2 * (1 + 1e-12) for a2, b2 in zip(est, est[1:]))
    prev = 1.0
    for j in range(info["outer_iters"]):
        assert est[j] <= prev * ir[j] * (1 + 1e-10) + 1e-15, (j, est[j], prev, ir[j])
        prev = ffom[j]


def test_level_to_the_eq5_tolerance_gives_one_top_step(cd2d):
    A, b = cd2d
    sv = _solver(A, max_outer=5)
    x, info = sv.solve(dev_vec(b), m=30, s=120, k=2, tol=1e-8, level_steps=[40])
    assert info["status"] == 0 and info["outer_iters"] == 1 and info["inner_reason"] == [3]
    assert info["inner_res"][0] <= 1e-8 * (1 + 1e-6)
    rel = np.linalg.norm(b - A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b)
    assert rel <= 1e-8


def test_multilevel_special_cases_and_arguments(cd2d):
    from paper_2506_18408_gb300 import sfgmres as py

    A, b = cd2d
    sv = _solver(A, max_outer=10)
    x, info = sv.solve(dev_vec(np.zeros(A.n)), m=20, s=80, k=2, level_steps=[3])  # b = 0 -> x = 0
    assert info["status"] == 0 and info["outer_iters"] == 0 and float(x.abs().max()) == 0.0
    for bad in ([], [0], [1025], [2, 2, 2, 2, 2]):
        with pytest.raises(py.SFGMRESError) as e:
            sv.solve(dev_vec(b), m=20, s=80, k=2, level_steps=bad)
        assert e.value.code == py.ERR_INVALID_ARG
    bn = b.copy()
    bn[3] = np.inf
    with pytest.raises(py.SFGMRESError) as e:
        sv.solve(dev_vec(bn), m=20, s=80, k=2, level_steps=[3])
    assert e.value.code == py.ERR_NAN
    _, info = sv.solve(dev_vec(b), m=20, s=80, k=2, level_steps=[3])  # the handle is still usable
    assert info["status"] == 0
