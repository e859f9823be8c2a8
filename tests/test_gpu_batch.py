"""GPU parity of the batched solver: many independent systems of uneven order, several right-hand sides each, solved
in lockstep by sfgmres_solve_batch, against the oracle run problem by problem on the same seeded inputs.

Each problem (system q, right-hand side r) is its own FGMRES / sGMRES solve with its own sketch, stop rules and
convergence test, so the bar is the single-system bar applied per problem: the recomputed relative residual
<= 1e-8 for both, outer counts within +-1, and the first Givens estimate within 1e-6 relative (FP64 inner).  Edge
cases: ragged systems that span several row blocks with a short last block, systems smaller than one block,
zero and non-finite right-hand sides inside a batch, the transposed batch, and invalid block-diagonal input.
"""
import numpy as np
import pytest

import workloads
from oracle import fgmres as ofg

from gpu_common import dev_vec, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _solver(A, **opt):
    from paper_2506_18408_gb300 import Solver

    return Solver(list(A.sys_n), A.row_ptr, A.col, A.val, sketch_seed=opt.pop("seed", 1), **opt)


def _per_problem(A, nrhs, b, x):
    """(system block, b_p, x_p) for every problem of the batch."""
    blocks = workloads.split_blocks(A)
    return [(blocks[q], b[a:a + n], x[a:a + n]) for q, a, n in workloads.problem_slices(A.sys_n, nrhs)]


def _rel_res(Aq, b, x):
    return float(np.linalg.norm(b - Aq.to_scipy() @ x) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def small():
    cfg = workloads.CONFIGS["batch_small"]
    A = cfg.build_matrix()
    b = cfg.build_rhs(A.n)
    return cfg, A, b


def test_batch_small_fp64_against_oracle(small):
    cfg, A, b = small
    sv = _solver(A, max_outer=cfg.max_outer, block_rows=512)  # several blocks per system, ragged last blocks
    x, info = sv.solve_batch(dev_vec(b), nrhs=cfg.nrhs, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol)
    x = x.cpu().numpy()
    assert info["status"] == 0 and info["problems"] == len(A.sys_n) * cfg.nrhs
    for p, (Aq, bp, xp) in enumerate(_per_problem(A, cfg.nrhs, b, x)):
        ref = ofg.fgmres(Aq.to_scipy(), bp, m=cfg.m, s=cfg.s, t=cfg.t, tol=cfg.tol, max_outer=cfg.max_outer)
        assert ref.status == ofg.CONVERGED
        assert info["status_p"][p] == 0
        assert _rel_res(Aq, bp, xp) <= cfg.tol, p
        assert abs(info["outer_iters_p"][p] - ref.outer_iters) <= 1, (p, info["outer_iters_p"][p], ref.outer_iters)
        assert abs(info["rel_res_true_p"][p] - ref.rel_res_true) <= cfg.tol


def test_batch_equals_single_system_solves(small):
    """A problem solved inside the batch gets the same outer count and residual history as on its own."""
    from paper_2506_18408_gb300 import Solver

    cfg, A, b = small
    sv = _solver(A, max_outer=cfg.max_outer)
    x, info = sv.solve_batch(dev_vec(b), nrhs=cfg.nrhs, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol)
    x = x.cpu().numpy()
    probs = _per_problem(A, cfg.nrhs, b, x)
    for p in (0, 7, len(probs) - 1):
        Aq, bp, xp = probs[p]
        one = Solver(Aq.n, Aq.row_ptr, Aq.col, Aq.val, sketch_seed=1, max_outer=cfg.max_outer)
        x1, i1 = one.solve(dev_vec(bp), m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol)
        assert abs(i1["outer_iters"] - info["outer_iters_p"][p]) <= 1
        # the same arithmetic up to the order of block partial sums (the row blocks differ): both are solutions to
        # 1e-8 relative residual of systems with condition numbers below 1e4
        assert np.linalg.norm(x1.cpu().numpy() - xp) <= 1e-4 * np.linalg.norm(xp)
        assert _rel_res(Aq, bp, x1.cpu().numpy()) <= cfg.tol


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_small_low_precision_inner_reaches_tol(small, prec):
    cfg, A, b = small
    sv = _solver(A, max_outer=cfg.max_outer, precision=prec)
    x, info = sv.solve_batch(dev_vec(b), nrhs=cfg.nrhs, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol)
    x = x.cpu().numpy()
    assert info["status"] == 0
    for Aq, bp, xp in _per_problem(A, cfg.nrhs, b, x):
        assert _rel_res(Aq, bp, xp) <= cfg.tol


def test_batch_transpose_matches_oracle_adjoint(small):
    cfg, A, b = small
    sv = _solver(A, max_outer=cfg.max_outer)
    x, info = sv.solve_batch(dev_vec(b), nrhs=cfg.nrhs, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol, transpose=True)
    x = x.cpu().numpy()
    assert info["status"] == 0
    for Aq, bp, xp in _per_problem(A, cfg.nrhs, b, x):
        At = Aq.to_scipy().T.tocsr()
        assert np.linalg.norm(bp - At @ xp) <= cfg.tol * np.linalg.norm(bp)


def test_batch_zero_and_nonfinite_right_hand_sides():
    from paper_2506_18408_gb300 import sfgmres as py

    A = workloads.block_diag([workloads.convdiff(N, (10.0, 5.0)) for N in (7, 33, 20)])
    nrhs = 2
    b = workloads.batch_rhs(A.sys_n, nrhs, seed=3)
    sl = workloads.problem_slices(A.sys_n, nrhs)
    q, a, n = sl[1]
    b[a:a + n] = 0.0                        # problem 1: b = 0 -> x = 0, OK
    q, a, n = sl[4]
    b[a + 3] = np.nan                       # problem 4: non-finite -> ERR_NAN for it alone
    x0 = workloads.rhs(A.n * nrhs, seed=8)  # nonzero initial guess everywhere
    sv = _solver(A, max_outer=50)
    with pytest.raises(py.SFGMRESError) as e:
        sv.solve_batch(dev_vec(b), dev_vec(x0), nrhs=nrhs, m=30, s=120, k=2, tol=1e-8)
    assert e.value.code == py.ERR_NAN
    # the per-problem outcomes: run again through the C call directly to read the statistics
    out = torch.empty(A.n * nrhs, dtype=torch.float64, device="cuda")
    st = py.BatchStats()
    P = len(sl)
    sa = (py.C.c_int32 * P)()
    st.status = py.C.cast(sa, py.C.POINTER(py.C.c_int32))
    bd, x0d = dev_vec(b), dev_vec(x0)  # keep the tensors alive across the call
    rc = py.load().sfgmres_solve_batch(sv.h, nrhs, bd.data_ptr(), x0d.data_ptr(), out.data_ptr(), 30, 120, 2, 1e-8,
                                       0, py.C.byref(st))
    assert rc == py.ERR_NAN
    status = list(sa)
    assert status[4] == py.ERR_NAN and status[1] == py.OK
    assert all(status[p] == py.OK for p in range(P) if p != 4)
    xo = out.cpu().numpy()
    blocks = workloads.split_blocks(A)
    for p, (q, a, n) in enumerate(sl):
        if p == 1:
            assert np.all(xo[a:a + n] == 0.0)
        elif p == 4:
            assert np.array_equal(xo[a:a + n], x0[a:a + n])
        else:
            assert _rel_res(blocks[q], b[a:a + n], xo[a:a + n]) <= 1e-8


def test_batch_tiny_and_single_row_systems():
    """Systems of order 1 and 2 and one that fills exactly one block."""
    mats = [workloads.convdiff(1, (3.0,)), workloads.convdiff(2, (1.0,)), workloads.convdiff(8, (4.0, 2.0)),
            workloads.random_zipf(300, seed=5)]
    A = workloads.block_diag(mats)
    b = workloads.batch_rhs(A.sys_n, 1, seed=4)
    sv = _solver(A, max_outer=60, block_rows=64)
    x, info = sv.solve_batch(dev_vec(b), nrhs=1, m=8, s=16, k=2, tol=1e-8)
    x = x.cpu().numpy()
    assert info["status"] == 0
    for Aq, bp, xp in _per_problem(A, 1, b, x):
        assert _rel_res(Aq, bp, xp) <= 1e-8


def test_batch_rejects_entries_outside_their_block_and_single_calls():
    from paper_2506_18408_gb300 import Solver
    from paper_2506_18408_gb300 import sfgmres as py

    A = workloads.block_diag([workloads.convdiff(5, (1.0, 1.0)), workloads.convdiff(4, (1.0, 1.0))])
    bad = A.col.copy()
    bad[3] = A.n - 1  # row 0 (system 0) pointing into system 1
    with pytest.raises(py.SFGMRESError) as e:
        Solver(list(A.sys_n), A.row_ptr, bad, A.val)
    assert e.value.code == py.ERR_INVALID_ARG
    sv = _solver(A)
    with pytest.raises(py.SFGMRESError) as e:
        sv.solve(dev_vec(np.ones(A.n)), m=4, s=16, k=2)
    assert e.value.code == py.ERR_INVALID_ARG
    with pytest.raises(py.SFGMRESError):
        sv.solve_batch(dev_vec(np.ones(A.n)), nrhs=0, m=4, s=16, k=2)


def test_graph_replay_and_eager_launches_give_identical_results(small):
    """Captured outer steps (first solve captures, second replays) and one-by-one launches run the same kernels in
    the same dependency order: the results agree bit for bit, for a batch and for a single system."""
    cfg, A, b = small
    for mat, nrhs, rhs in ((A, cfg.nrhs, b), (workloads.convdiff(64, (20.0, 10.0)), 1, workloads.rhs(4096, seed=0))):
        if mat.sys_n is None:
            from paper_2506_18408_gb300 import Solver

            sv = Solver(mat.n, mat.row_ptr, mat.col, mat.val, sketch_seed=1, max_outer=20)
        else:
            sv = _solver(mat, max_outer=cfg.max_outer)
        outs = []
        for graph in (1, 1, 0):
            sv.set("graph", graph)
            if nrhs == 1 and mat.sys_n is None:
                x, info = sv.solve(dev_vec(rhs), m=30, s=120, k=2, tol=1e-8)
                outs.append((x.cpu().numpy(), info["outer_iters"], info["inner_k"]))
            else:
                x, info = sv.solve_batch(dev_vec(rhs), nrhs=nrhs, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol)
                outs.append((x.cpu().numpy(), info["outer_iters_p"], None))
            assert info["status"] == 0
        for x, it, ks in outs[1:]:
            assert np.array_equal(x, outs[0][0])
            assert it == outs[0][1] and ks == outs[0][2]


def test_autotune_picks_a_valid_shape_and_solves_stay_correct(small):
    cfg, A, b = small
    sv = _solver(A, max_outer=cfg.max_outer)
    br, vec, step_ms = sv.autotune(nrhs=cfg.nrhs, m=cfg.m, s=cfg.s, k=cfg.t)
    assert 256 <= br <= 8192 and br % 32 == 0 and step_ms > 0
    assert sv.get("block_rows") == br
    x, info = sv.solve_batch(dev_vec(b), nrhs=cfg.nrhs, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol)
    x = x.cpu().numpy()
    assert info["status"] == 0
    for Aq, bp, xp in _per_problem(A, cfg.nrhs, b, x):
        assert _rel_res(Aq, bp, xp) <= cfg.tol
    Z = workloads.random_zipf(30_000, seed=3)  # long rows: the SpMV width is tuned too
    from paper_2506_18408_gb300 import Solver

    sz = Solver(Z.n, Z.row_ptr, Z.col, Z.val, sketch_seed=1)
    br, vec, _ = sz.autotune(m=20, s=80, k=4)
    assert vec in (0, 1, 2, 4, 8, 16, 32)  # 0 = the length-binned SpMV
    bz = workloads.rhs(Z.n, seed=1)
    xz, iz = sz.solve(dev_vec(bz), m=20, s=80, k=4, tol=1e-8)
    assert iz["status"] == 0 and _rel_res(Z, bz, xz.cpu().numpy()) <= 1e-8


def test_profiled_solves_time_the_working_launches_with_and_without_graphs():
    """Profiling puts the kernel timing events into the captured graphs: a profiled solve gives the same result as an
    unprofiled one, with graphs (captured, then replayed) and without, and counts exactly the inner steps that built
    a basis vector (the sum of k_j over the outer steps)."""
    from paper_2506_18408_gb300 import Solver

    mat = workloads.convdiff(64, (20.0, 10.0))
    rhs = workloads.rhs(mat.n, seed=0)
    sv = Solver(mat.n, mat.row_ptr, mat.col, mat.val, sketch_seed=1, max_outer=20)
    sv.set("fused_step", 0)  # the two kernels of a step, timed separately
    bd = dev_vec(rhs)
    x_ref, info_ref = sv.solve(bd, m=30, s=120, k=2, tol=1e-8)
    assert info_ref["status"] == 0 and info_ref["n_inner_spmv"] == 0
    for graph in (1, 1, 0):
        sv.set("graph", graph)
        sv.set("profile", 1)
        x, info = sv.solve(bd, m=30, s=120, k=2, tol=1e-8)
        sv.set("profile", 0)
        assert info["status"] == 0
        assert np.array_equal(x.cpu().numpy(), x_ref.cpu().numpy())
        steps = int(sum(info["inner_k"]))
        assert steps == info["total_inner"] == info_ref["total_inner"]
        for key in ("inner_spmv", "inner_axpy", "qr"):
            assert info["n_" + key] == steps
            assert 0.0 < info["t_%s_ms" % key] < info["t_total_ms"]


def test_cycle_span_profile_times_full_cycles_only():
    """Profile mode 2 records one pair of events around each inner cycle's chain of m step launches: the solve is
    bit for bit the unprofiled one (graphs captured, replayed, and off), the spans cover exactly the cycles whose m
    steps all built a basis vector, and their sum lies inside the solve's time."""
    from paper_2506_18408_gb300 import Solver

    mat = workloads.convdiff(64, (20.0, 10.0))
    bd = dev_vec(workloads.rhs(mat.n, seed=0))
    sv = Solver(mat.n, mat.row_ptr, mat.col, mat.val, sketch_seed=1, max_outer=80)
    x_ref, info_ref = sv.solve(bd, m=10, s=60, k=2, tol=1e-8)
    assert info_ref["status"] == 0 and info_ref["n_step_span"] == 0
    full = sum(1 for k in info_ref["inner_k"] if k == 10)
    assert full > 0
    for graph in (1, 1, 0):
        sv.set("graph", graph)
        sv.set("profile", 2)
        x, info = sv.solve(bd, m=10, s=60, k=2, tol=1e-8)
        sv.set("profile", 0)
        assert info["status"] == 0
        assert np.array_equal(x.cpu().numpy(), x_ref.cpu().numpy())
        assert info["inner_k"] == info_ref["inner_k"]
        assert info["n_step_span"] == 10 * full
        assert info["n_inner_spmv"] == 0
        assert 0.0 < info["t_step_span_ms"] < info["t_total_ms"]
    sv.close()


def test_fused_inner_step_matches_the_two_kernel_step():
    """One launch per inner step (the inner SpMV kernel's work, a grid-wide arrival, then the Arnoldi update of the
    CTA's own rows) runs the same arithmetic in the same order as the two kernels: FP64 and FP32-inner solves agree
    bit for bit with and without graphs, and profiling shows the fused path was taken (no separate update launches)."""
    from paper_2506_18408_gb300 import Solver

    mat = workloads.convdiff(64, (20.0, 10.0))
    rhs = workloads.rhs(mat.n, seed=0)
    bd = dev_vec(rhs)
    for prec in ("fp64", "fp32"):
        sv = Solver(mat.n, mat.row_ptr, mat.col, mat.val, sketch_seed=1, max_outer=20, precision=prec)
        assert int(sv.get("fused_step")) == 1
        sv.set("fused_step", 0)
        x_two, info_two = sv.solve(bd, m=30, s=120, k=2, tol=1e-8)
        assert info_two["status"] == 0
        sv.set("fused_step", 1)
        for graph in (1, 1, 0):
            sv.set("graph", graph)
            x, info = sv.solve(bd, m=30, s=120, k=2, tol=1e-8)
            assert info["status"] == 0
            assert np.array_equal(x.cpu().numpy(), x_two.cpu().numpy())
            assert info["inner_k"] == info_two["inner_k"]
        sv.set("profile", 1)
        _, ip = sv.solve(bd, m=30, s=120, k=2, tol=1e-8)
        assert ip["n_inner_axpy"] == 0 and ip["n_inner_spmv"] == ip["total_inner"] > 0
        sv.set("profile", 0)
        sv.set("fused_step", 0)
        sv.set("profile", 1)
        _, ip2 = sv.solve(bd, m=30, s=120, k=2, tol=1e-8)
        assert ip2["n_inner_axpy"] == ip2["total_inner"]
        sv.close()


def test_fused_step_wait_that_gives_up_is_reported_and_the_handle_stays_usable():
    """The fused step's grid-wide wait is bounded: made to wait for one arrival that never comes, the first wait of
    the cycle gives up after its polls (about a second), the later ones return at once, and the solve reports
    SFGMRES_ERR_CUDA instead of hanging; with the hook off again the same handle solves normally, bit for bit as
    before."""
    from paper_2506_18408_gb300 import Solver
    from paper_2506_18408_gb300.sfgmres import SFGMRESError

    mat = workloads.convdiff(64, (20.0, 10.0))
    bd = dev_vec(workloads.rhs(mat.n, seed=0))
    sv = Solver(mat.n, mat.row_ptr, mat.col, mat.val, sketch_seed=1, max_outer=20)
    x_ref, info_ref = sv.solve(bd, m=30, s=120, k=2, tol=1e-8)
    assert info_ref["status"] == 0
    sv.set("step_wait_extra", 1)
    with pytest.raises(SFGMRESError) as ei:
        sv.solve(bd, m=30, s=120, k=2, tol=1e-8)
    assert ei.value.code == -2 and "gave up" in str(ei.value)
    sv.set("step_wait_extra", 0)
    x, info = sv.solve(bd, m=30, s=120, k=2, tol=1e-8)
    assert info["status"] == 0 and np.array_equal(x.cpu().numpy(), x_ref.cpu().numpy())
    sv.close()
