"""The paper's preferred setting on the GPU (Section 4.1, the truncation sweep): a Clarkson-Woodruff sketch (one +-1 per
column, zeta = 1), s = 2 k_max = 1000, k_max = 500, the inner length decided by the condition number of the sketched
basis (rule C2, C3 off) and the truncation t = 0..5, against the oracle on the same seeded inputs (3D
convection-diffusion 24^3, n = 13,824).

Rule C2 evaluates the proxy max|r_ll| / min|r_ll| of the sketched QR.  For the power basis (t = 0) and t = 1 the proxy
first grows by a factor of about 2-3 per step (1e8 after ~18 steps for t = 0, 1e10 after ~22) and then reaches a
plateau a little below 1e15 on which the smallest |r_ll| is set by rounding (about u max|r_ll|) and fluctuates for a
hundred steps or more; where such a cycle crosses 1e15 is decided by rounding noise (the same oracle ends its first
t = 0 cycle after 167 steps on one CPU and after 146 on another, and the GPU, whose basis and sketch carry less
rounding, later still).  So:

* the C2 mechanism is compared step for step at a threshold on the steep part of the curve, 1e10: the GPU's cycle
  lengths equal the oracle's for every cycle but the last (within one step there), and the outer iteration counts
  agree within 1;
* at the paper's threshold 1e15 the checks are the ones rounding does not decide: FGMRES converges to 1e-8 for every
  t (Section 4.1: it converges even for the power basis); t = 0 and t = 1 end every cycle by C2 before k_max; t >= 2
  keeps the basis well conditioned up to k_max, one cycle of all 500 columns (rule C1, the sketched QR at full width:
  i up to 499 against Q of 1000 x 500) solves the system on both sides; and the first cycle gets no shorter as t
  grows (larger t, better conditioned bases, longer cycles).
"""
import numpy as np
import pytest

import workloads
from oracle import fgmres as ofg

from gpu_common import dev_vec, need_gpu

pytestmark = pytest.mark.gpu

M, S, ZETA = 500, 1000, 1


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def problem():
    A = workloads.convdiff(24, (50.0, 30.0, 10.0))
    return A, workloads.rhs(A.n, seed=0)


def _run(problem, t, thr):
    from paper_2506_18408_gb300 import Solver

    A, b = problem
    As = A.to_scipy()
    sv = Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=1, zeta=ZETA, c3=0, max_outer=60, cond_threshold=thr)
    x, info = sv.solve(dev_vec(b), m=M, s=S, k=t, tol=1e-8)
    sv.close()
    ref = ofg.fgmres(As, b, None, m=M, s=S, t=t, tol=1e-8, max_outer=60, c3=False, zeta=ZETA, cond_thr=thr)
    rel = float(np.linalg.norm(b - As @ x.cpu().numpy()) / np.linalg.norm(b))
    print(f"thr={thr:.0e} t={t}: GPU outer {info['outer_iters']} k {info['inner_k']} | oracle outer "
          f"{ref.outer_iters} k {ref.inner_k}")
    return info, ref, rel


@pytest.mark.parametrize("t", [0, 1])
def test_c2_driven_cycle_lengths_match_oracle(problem, t):
    info, ref, rel = _run(problem, t, 1e10)
    assert info["status"] == 0 and ref.status == ofg.CONVERGED
    assert rel <= 1e-8 and ref.rel_res_true <= 1e-8
    assert set(info["inner_reason"]) == {2} == set(ref.inner_reason)
    assert abs(info["outer_iters"] - ref.outer_iters) <= 1
    # every cycle but the last has the oracle's length; the last cycle starts from an outer vector v_j carrying the
    # rounding of all earlier outer steps, so its C2 decision may fall one step apart
    common = min(len(info["inner_k"]), len(ref.inner_k))
    assert info["inner_k"][:common - 1] == ref.inner_k[:common - 1]
    assert abs(info["inner_k"][common - 1] - ref.inner_k[common - 1]) <= 1


@pytest.fixture(scope="module")
def sweep_1e15(problem):
    return {t: _run(problem, t, 1e15) for t in range(6)}


@pytest.mark.parametrize("t", range(6))
def test_paper_threshold_sweep(sweep_1e15, t):
    info, ref, rel = sweep_1e15[t]
    assert info["status"] == 0 and ref.status == ofg.CONVERGED
    assert rel <= 1e-8 and ref.rel_res_true <= 1e-8
    if t <= 1:
        assert set(info["inner_reason"]) == {2} == set(ref.inner_reason)
        assert all(k < M for k in info["inner_k"])
    else:
        assert info["inner_k"] == [M] == ref.inner_k and info["inner_reason"] == [1] == ref.inner_reason


def test_first_cycle_length_nondecreasing_in_t(sweep_1e15):
    first = [sweep_1e15[t][0]["inner_k"][0] for t in range(6)]
    assert all(a <= b for a, b in zip(first, first[1:])), first
