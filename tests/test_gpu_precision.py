"""Precision-matched GPU parity of the FP32-inner and BF16-basis forms against the oracle's matching inner modes.

The inner sGMRES cycle runs in FP32 (matrix values, basis, dot products, sketch and their accumulation), or in FP32
with every stored basis vector rounded to BF16; the outer FGMRES, the sketched QR and least squares, z = B y and the
recomputed residual stay FP64 (Section 3: the inner cycle is only a variable preconditioner, and the FP64 outer
FGMRES of Algorithm 1 keeps the accuracy).  The oracle's ``inner="fp32"`` / ``"bf16"`` modes round the same
quantities, in NumPy, in the paper's order; these tests compare the CUDA path with them on the same seeded inputs.

Tolerances, with eps32 = 2^-24 and the BF16 unit u16 = 2^-8:

* FP32 first-cycle basis vector b_l (l = 0, 1, ...): the GPU and the oracle evaluate every inner step in FP32 with
  different summation orders (rows of up to 256 products, dot products and sketch sums over n terms in block partials
  vs. NumPy's pairwise sums), so one step's results differ by up to a few hundred eps32 relative, amplified by the
  normalisation 1/eta_l; the truncated recurrence carries earlier differences forward, about linearly along the
  cycle (the oracle's own FP32-vs-FP64 distance is at most 10 (l+1) eps32 on these workloads).  Bound:
  ||b_l^gpu - b_l^oracle|| <= 256 (l+1) eps32 ||b_l^oracle||.
* BF16 basis: each stored vector is rounded to 8 significant bits.  The GPU rounds the vector scaled by a power of two,
  the oracle the normalised vector (a different significand), so the two roundings are independent: up to 2^-8
  relative per stored vector (twice the 2^-9 rounding bound), carried forward by the recurrence.  Bound:
  u16 (1 + l/2).
* The cycle's correction z: compared through the inner residual ||v - A z||: within 2^-12 relative (FP32) or 2^-5
  (BF16) of the oracle's, plus 2 delta kappa(S A B_k), the change of a least-squares residual under a relative
  perturbation delta (256 eps32, or u16) of its matrix, which matters for the ill-conditioned power basis (t = 0).
* Full solves (both sides FP64 outside the cycle): both reach the recomputed 1e-8 residual; outer iteration counts
  within +-1 (FP32) and +-2 (BF16).  The first outer step's residual estimate is beta times the first cycle's inner
  residual, so it carries one cycle's worth of inner rounding differences: FP64 within 1e-6 relative, FP32 within 2^-8
  (the first-order bound delta ||S A B_k|| ||y_k|| / rho_k is of order one for the 60- and 100-column cycles of the
  full-size workloads, kappa(S A B_k) ~ 7e4; the differences measured there are about 1e-3, and an FP32 oracle differs
  from the FP64 oracle by as much), BF16 within 2^-4.  The inner lengths of the leading cycles that the oracle ended
  by rule C1 and that start from a residual above 10 tol agree for FP64 and FP32 (closer to tol, rule C3 can end a
  cycle as soon as its sketched residual falls below tol / ||r~_{j-1}|| > 0.1, a point that moves with the rounding);
  with a BF16 basis the estimates that decide rule C3 drift apart by the 8-bit noise, so only counts and residuals
  are compared.  With a BF16 basis each outer step reduces the
  residual by about the accuracy of the 8-bit basis, so which of two close steps meets 1e-8 depends on the roundings:
  the GPU's storage (the vector scaled by a power of two) and the oracle's (the normalised vector) round
  independently, and on the 12-system batch that alone moves single counts by up to 2 (an oracle copy storing the
  scaled vector instead gave differences of -2..+2 over the 36 problems); the batch's total outer steps must agree
  within 10 %.

The full-size oracle solves (128^3 and the random Zipf matrix, n = 2M) come from ``tests/golden/oracle_runs.json``,
written by ``tests/golden/make_oracle_runs.py`` from the oracle alone on the same seeded inputs.
"""
import json
import os

import numpy as np
import pytest

import workloads
from oracle import fgmres as ofg
from oracle import sgmres as osg
from oracle import sketch as osk

from gpu_common import dev_vec, need_gpu, rel_err, torch

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
U16 = 2.0 ** -8
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_runs.json")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def basis_tol(prec: str, l: int) -> float:
    return 256 * (l + 1) * EPS32 if prec == "fp32" else U16 * (1 + l / 2)


def _solver(A, **opt):
    from paper_2506_18408_gb300 import Solver

    return Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=opt.pop("seed", 1), **opt)


def _first_cycle(sv, A, prec, m, s, t, steps=None):
    """GPU first cycle on v = b/||b|| against the oracle's cycle in the same inner precision (C1/C2 only)."""
    steps = steps or m
    b = workloads.rhs(A.n, seed=0)
    v = b / np.linalg.norm(b)
    z, k, reason, B, _ = sv.inner_cycle(dev_vec(v), m=steps, s=s, k=t)
    As = A.to_scipy()
    S = osk.sketch_matrix(A.n, s, 8, 1)
    ref = osg.sgmres_cycle(As, v, S, steps, t, record=True, inner=prec)
    assert (k, reason) == (ref.k, ref.reason)
    B = B.cpu().numpy()
    errs = []
    for l in range(len(ref.basis)):
        e = rel_err(B[l], ref.basis[l])
        errs.append(e)
        assert e <= basis_tol(prec, l), (prec, l, e, basis_tol(prec, l))
    zh = z.cpu().numpy()
    rg = np.linalg.norm(v - As @ zh)
    ro = np.linalg.norm(v - As @ ref.z)
    # the sketched least squares turns a relative perturbation delta of S A B_k (delta = 256 eps32 in FP32, u16 with
    # a BF16 basis) into a change of its residual of up to about 2 delta kappa(S A B_k) ||S v|| (||S v|| ~ 1)
    delta = 256 * EPS32 if prec == "fp32" else U16
    kappa = np.linalg.cond(ref.sab)
    assert abs(rg - ro) <= (2.0 ** -12 if prec == "fp32" else 2.0 ** -5) * ro + 2 * delta * kappa, (prec, rg, ro, kappa)
    return errs, zh, ref, B


CYCLE_CASES = [
    ("cd2d_64", workloads.CONFIGS["cd2d_64"].build_matrix, 30, 120, 2),
    ("zipf_20011_t4", lambda: workloads.random_zipf(20_011, seed=1), 40, 160, 4),
    ("cd3d_17_t1", lambda: workloads.convdiff(17, (50.0, 30.0, 10.0)), 30, 120, 1),
    ("cd2d_37_t0", lambda: workloads.convdiff(37, (20.0, 10.0)), 12, 100, 0),
]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("name,make,m,s,t", CYCLE_CASES, ids=[c[0] for c in CYCLE_CASES])
def test_first_cycle_basis_low_precision(name, make, m, s, t, prec):
    A = make()
    sv = _solver(A, precision=prec)
    errs = _first_cycle(sv, A, prec, m, s, t)[0]
    print(f"{name} {prec}: max basis error vs the oracle's {prec} cycle {max(errs):.2e}")


@pytest.fixture(scope="module")
def cd3d():
    cfg = workloads.CONFIGS["cd3d_128"]
    A = cfg.build_matrix()
    return cfg, A, cfg.build_rhs(A.n)


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_cd3d_128_first_cycle_low_precision(cd3d, prec):
    """The 128^3 workload in the launch configuration of the solve (row blocks, fused step): 12 inner steps of the
    first cycle against the oracle's cycle in the same precision, and the distance of each basis vector from the
    FP64 oracle's (the error of the precision form itself, bounded like the FP32 form's drift)."""
    cfg, A, _ = cd3d
    sv = _solver(A, precision=prec, seed=cfg.sketch_seed)
    errs, zh, _, B = _first_cycle(sv, A, prec, cfg.m, cfg.s, cfg.t, steps=12)
    b = workloads.rhs(A.n, seed=0)
    v = b / np.linalg.norm(b)
    ref64 = osg.sgmres_cycle(A.to_scipy(), v, osk.sketch_matrix(A.n, cfg.s, 8, 1), 12, cfg.t, record=True)
    e64 = [rel_err(B[l], ref64.basis[l]) for l in range(len(ref64.basis))]
    for l, e in enumerate(e64):
        assert e <= basis_tol(prec, l), (l, e)
    print(f"cd3d_128 {prec}: basis vs oracle {prec} max {max(errs):.2e}; vs oracle fp64 max {max(e64):.2e}; "
          f"z vs fp64 {rel_err(zh, ref64.z):.2e}")


def _check_solve_against_golden(info, rel, g, est_tol, count_tol=1):
    assert info["status"] == 0 and g["status"] == 0
    assert rel <= g["tol"] and g["rel_res_true"] <= g["tol"]
    assert abs(info["outer_iters"] - g["outer_iters"]) <= count_tol, (info["outer_iters"], g["outer_iters"])
    est = info["res_est"]
    assert all(b2 <= a2 * (1 + 1e-12) for a2, b2 in zip(est, est[1:])), est  # non-increasing (Algorithm 1)
    assert abs(est[0] - g["est_hist"][0]) <= est_tol * g["est_hist"][0], (est[0], g["est_hist"][0])
    if g["inner"] == "bf16":
        return
    # the leading cycles that the oracle ended by rule C1 (k = m) have the same length on the GPU, as long as they start
    # from a residual above 10 tol: rule C3 (the Eq. 5 bound ||r~_{j-1}|| rho_k against tol ||b||) can end a cycle
    # that starts closer to tol as soon as its sketched residual rho_k falls below tol ||b|| / ||r~_{j-1}|| > 0.1,
    # which these 60-step cycles reach, and where it fires then depends on the rounding of the low-precision cycles
    start = [g["est_hist"][j - 1] if j > 0 else np.inf for j in range(len(g["inner_reason"]))]
    lead = next((j for j, r in enumerate(g["inner_reason"]) if r != 1 or start[j] <= 10 * g["tol"]),
                len(g["inner_reason"]))
    print("GPU inner_k", info["inner_k"], "reasons", info["inner_reason"], "est", ["%.3e" % e for e in est])
    assert info["inner_k"][:lead] == g["inner_k"][:lead], (info["inner_k"], g["inner_k"])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_cd3d_128_low_precision_solve_against_oracle(cd3d, golden, prec):
    cfg, A, b = cd3d
    g = golden[f"cd3d_128_{prec}"]
    assert (g["n"], g["m"], g["s"], g["t"]) == (A.n, cfg.m, cfg.s, cfg.t)
    sv = _solver(A, precision=prec, seed=cfg.sketch_seed, max_outer=cfg.max_outer)
    x, info = sv.solve(dev_vec(b), m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol)
    xh = x.cpu().numpy()
    As = A.to_scipy()
    rel = float(np.linalg.norm(b - As @ xh) / np.linalg.norm(b))
    _check_solve_against_golden(info, rel, g, 2.0 ** -8 if prec == "fp32" else 2.0 ** -4, 1 if prec == "fp32" else 2)
    print(f"cd3d_128 {prec}: outer {info['outer_iters']} (oracle {g['outer_iters']}), rel_res {rel:.2e}")


@pytest.fixture(scope="module")
def zipf():
    cfg = workloads.CONFIGS["zipf_2m"]
    A = cfg.build_matrix()
    return cfg, A, cfg.build_rhs(A.n)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_zipf_2m_solve_against_oracle(zipf, golden, prec):
    """The random Zipf matrix (n = 2M, t = 4, s = 240, length-binned SpMV) solved to 1e-8 against the oracle's full
    solve in the same inner precision: outer counts within 1, the same lengths for the cycles the oracle ended by rule
    C1, and the residual estimates of every step both runs take within 1e-6 relative plus 1e-11 ||b|| (FP64), or the
    first within 2^-8 (FP32)."""
    cfg, A, b = zipf
    g = golden[f"zipf_2m_{prec}"]
    assert (g["n"], g["nnz"], g["m"], g["s"], g["t"]) == (A.n, A.nnz, cfg.m, cfg.s, cfg.t)
    sv = _solver(A, precision=prec, seed=cfg.sketch_seed, max_outer=cfg.max_outer)
    x, info = sv.solve(dev_vec(b), m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol)
    xh = x.cpu().numpy()
    rel = float(np.linalg.norm(b - A.to_scipy() @ xh) / np.linalg.norm(b))
    _check_solve_against_golden(info, rel, g, 1e-6 if prec == "fp64" else 2.0 ** -8)
    if prec == "fp64":
        # 1e-6 relative, with an absolute floor (in units of ||b||) of kappa(S A B_k) u64 ~ 7.6e4 * 1.1e-16 ~ 1e-11: each
        # correction z_j carries rounding differences of that relative size, which dominate once the estimate is
        # near the 1e-8 target
        est = info["res_est"]
        for j in range(min(len(est), len(g["est_hist"])) - 1):
            assert abs(est[j] - g["est_hist"][j]) <= 1e-6 * g["est_hist"][j] + 1e-11, (j, est[j], g["est_hist"][j])
    print(f"zipf_2m {prec}: outer {info['outer_iters']} (oracle {g['outer_iters']}), rel_res {rel:.2e}")


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_small_low_precision_outer_counts_match_oracle(prec):
    """Every problem of the 12-system batch (ragged sizes, 3 right-hand sides) in FP32-inner / BF16-basis mode
    against the oracle's solve of that problem in the same inner precision: both reach 1e-8, outer counts within 1
    (FP32) or 2 (BF16), and the batch's total outer steps within 10 %."""
    from paper_2506_18408_gb300 import Solver

    cfg = workloads.CONFIGS["batch_small"]
    A = cfg.build_matrix()
    b = cfg.build_rhs(A.n)
    sv = Solver(list(A.sys_n), A.row_ptr, A.col, A.val, sketch_seed=1, max_outer=cfg.max_outer, precision=prec)
    x, info = sv.solve_batch(dev_vec(b), nrhs=cfg.nrhs, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol)
    x = x.cpu().numpy()
    assert info["status"] == 0
    blocks = workloads.split_blocks(A)
    count_tol = 1 if prec == "fp32" else 2
    tot_gpu = tot_ref = 0
    for p, (q, a, nq) in enumerate(workloads.problem_slices(A.sys_n, cfg.nrhs)):
        Aq = blocks[q].to_scipy()
        bp = b[a:a + nq]
        ref = ofg.fgmres(Aq, bp, m=cfg.m, s=cfg.s, t=cfg.t, tol=cfg.tol, max_outer=cfg.max_outer, inner=prec)
        assert ref.status == ofg.CONVERGED
        assert np.linalg.norm(bp - Aq @ x[a:a + nq]) <= cfg.tol * np.linalg.norm(bp)
        got = info["outer_iters_p"][p]
        assert abs(got - ref.outer_iters) <= count_tol, (p, got, ref.outer_iters)
        tot_gpu += got
        tot_ref += ref.outer_iters
    assert abs(tot_gpu - tot_ref) <= 0.1 * tot_ref, (tot_gpu, tot_ref)
    print(f"batch_small {prec}: outer steps over the batch {tot_gpu} (oracle {tot_ref})")
