"""Benchmark: time to a 1e-8 relative residual of sketched FGMRES on one GB300.

A step is one full solve (every step of the method: residual, inner sGMRES cycles, outer FGMRES steps, final
iterate and recomputed true residual) of the 3D convection-diffusion system on a 128^3 grid (n = 2,097,152,
nnz = 14,581,760; beta = (50, 30, 10); b ~ N(0,1) seed 0; inner m = 100, truncation k = 2, sketch s = 400 with 8
nonzeros per column, seed 1; tol 1e-8), with b and A resident in HBM.  The headline is the plain FP64 solver; the
FP32-inner and BF16-basis forms are reported beside it on the same inputs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--profile-case [cd3d_128|zipf_2m|qr_cd3d|cd2d_64]]

``--impl reference`` times the CPU oracle (plain FP64 NumPy/SciPy restatement of the method) on a bounded sample
of the same workload.  ``--profile-case`` runs short solves for ncu captures and prints nothing else.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "time to 1e-8 rel. residual; inner-cycle HBM GB/s vs peak; FP32-inner vs FP64"
CFG = workloads.CONFIGS["cd3d_128"]
WORKLOAD = ("cd3d_128: 3D convection-diffusion 128^3, upwind 7-point, beta=(50,30,10), b~N(0,1) seed 0, x0=0; "
            "inner sGMRES m=100, k(truncation)=2, sparse-sign sketch s=400 zeta=8 seed 1; FGMRES tol 1e-8")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"sfgmres_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def alg_bytes_inner_spmv(n, nnz, t, zeta, s, nblk, sv):
    """Compulsory bytes of one fused inner SpMV + dots + sketch launch: A (values, column indices, row pointers), b_i
    gathered once, the t - 1 older window vectors, w written, the sketch gather lists and segment table, and the
    per-block partials."""
    a = nnz * (sv + 4) + 4 * (n + 1)          # CSR values + column indices + row pointers
    vec = n * sv * (1 + max(t - 1, 0)) + n * sv  # b_i (gathered once) + older window vectors + w written
    sk = 2 * n * zeta + 4 * (nblk * s + 1) + sv * nblk * (s + t)  # gather lists, segment table, partials
    return a + vec + sk


def alg_bytes_solve(n, nnz, t, sv, sval, inner_steps, outer_steps):
    """Compulsory bytes of a whole solve of one problem: its inner steps (alg_bytes_inner_step), each cycle's z = B y
    ((k + 1) n S_v read, n FP64 written, summed over the cycles: (inner_steps + outer_steps) n S_v + 8 n per cycle), and
    each outer step j (an FP64 SpMV with A and z_j read, w written, and CGS2 against v_0..v_j: (4 j + 3) n 8)."""
    inner = inner_steps * alg_bytes_inner_step_prec(n, nnz, t, sv, sval)
    gemv = (inner_steps + outer_steps) * n * sv + outer_steps * 8 * n
    outer = sum(nnz * 12 + 4 * (n + 1) + 16 * n + (4 * j + 3) * n * 8 for j in range(outer_steps))
    return inner + gemv + outer


def alg_bytes_inner_step_prec(n, nnz, t, sv, sval):
    """alg_bytes_inner_step with the matrix values in sval bytes (FP32 copy for FP32 inner cycles)."""
    return nnz * (sval + 4) + 4 * (n + 1) + (2 * t + 3) * n * sv


def alg_bytes_inner_step(n, nnz, t, sv):
    """Compulsory bytes of one whole inner step (fused SpMV + dots + sketch, Arnoldi update; the sketch hashed, so no
    bytes for S): A once, b_i read, w written and read back, t window vectors read for the update, t - 1 of them
    again for the dots, b_{i+1} written."""
    return nnz * (sv + 4) + 4 * (n + 1) + (2 * t + 3) * n * sv


def max_over_ranks(dist, value: float, device) -> float:
    """The largest of every rank's ``value`` (each rank calls it with one float); ``value`` itself without a
    process group."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch

    from paper_2506_18408_gb300 import Solver, build

    build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    A = CFG.build_matrix()
    b = CFG.build_rhs(A.n)
    n, nnz = A.n, A.nnz
    stream = torch.cuda.current_stream()
    solver = Solver(n, A.row_ptr, A.col, A.val, sketch_seed=CFG.sketch_seed, zeta=CFG.zeta,
                    max_outer=CFG.max_outer, stream=stream.cuda_stream)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.empty_like(bd)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2 (129 MB)

    if args.profile_case == "zipf_2m":
        # the random Zipf matrix (length-binned SpMV), FP64 then FP32 inner, m = 20, two outer steps
        solver.close()
        zc = workloads.CONFIGS["zipf_2m"]
        Z = zc.build_matrix()
        zb = torch.from_numpy(zc.build_rhs(Z.n)).to(dev)
        zs = Solver(Z.n, Z.row_ptr, Z.col, Z.val, sketch_seed=zc.sketch_seed, max_outer=2, stream=stream.cuda_stream)
        for prec in ("fp64", "fp32"):
            zs.set("precision", prec)
            zs.solve(zb, m=20, s=zc.s, k=zc.t, tol=zc.tol)
        torch.cuda.synchronize()
        zs.close()
        return
    if args.profile_case == "cd2d_64":
        # the small 2D workload (latency bound): one warm-up solve (sketch lists, graphs), then one full FP64 solve
        solver.close()
        sc = workloads.CONFIGS["cd2d_64"]
        S2 = sc.build_matrix()
        sb = torch.from_numpy(sc.build_rhs(S2.n)).to(dev)
        ss = Solver(S2.n, S2.row_ptr, S2.col, S2.val, sketch_seed=sc.sketch_seed, zeta=sc.zeta, max_outer=sc.max_outer,
                    stream=stream.cuda_stream)
        for _ in range(2):
            ss.solve(sb, m=sc.m, s=sc.s, k=sc.t, tol=sc.tol)
        torch.cuda.synchronize()
        ss.close()
        return
    if args.profile_case == "qr_cd3d":
        # one full inner cycle (m = 100, C3 off: sketched-QR updates i = 0..99) of the same workload
        solver.set("max_outer", 1)
        solver.set("c3", 0)
        solver.solve(bd, m=CFG.m, s=CFG.s, k=CFG.t, tol=CFG.tol, out=xd)
        torch.cuda.synchronize()
        return
    if args.profile_case:
        # same matrix, sketch and kernels; a short basis (m = 20) and two outer steps keep the device footprint
        # (~0.6 GB) and the launch count small for ncu
        solver.set("max_outer", 2)
        for prec in ("fp64", "fp32"):
            solver.set("precision", prec)
            solver.solve(bd, m=20, s=CFG.s, k=CFG.t, tol=CFG.tol, out=xd)
        torch.cuda.synchronize()
        return

    def timed(precision, K, W, profile=0):
        solver.set("precision", precision)
        solver.set("profile", 0)
        for _ in range(W):
            solver.solve(bd, m=CFG.m, s=CFG.s, k=CFG.t, tol=CFG.tol, out=xd)
        solver.set("profile", int(profile))
        times, infos = [], []
        for _ in range(K):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            _, info = solver.solve(bd, m=CFG.m, s=CFG.s, k=CFG.t, tol=CFG.tol, out=xd)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            infos.append(info)
        solver.set("profile", 0)
        return times, infos

    with ClockSampler(local) as clk:
        t64, i64 = timed("fp64", args.steps, args.warmup)
        # the same solves with the kernels bracketed by CUDA events (event nodes in the captured graphs), for the
        # roofline; the events lengthen the solve, so the headline time comes from the unprofiled solves above.
        # Events around every launch (the events' own cost included):
        tp, ip = timed("fp64", max(3, args.steps // 2), 1, profile=1)
        # one pair of events around each full inner cycle's chain of m step launches: no event between two launches,
        # so the span per launch includes the gaps between them but no event's own cost
        ts, isp = timed("fp64", max(3, args.steps // 2), 1, profile=2)
    t32, i32 = timed("fp32", args.steps, max(3, args.warmup // 2))
    t16, i16 = timed("bf16", args.steps, max(3, args.warmup // 2))
    sec = max_over_ranks(dist, statistics.mean(t64), dev)

    # end to end through the public API with pinned host buffers (copies inside the timed region)
    solver.set("precision", "fp64")
    bh = torch.empty(n, dtype=torch.float64, pin_memory=True)
    bh.numpy()[:] = b
    xh = torch.empty(n, dtype=torch.float64, pin_memory=True)
    # untimed warm-up: switching back to FP64 changed the row-block geometry (sketch lists and graphs are rebuilt)
    for _ in range(max(1, args.warmup)):
        solver.solve(bh.numpy(), m=CFG.m, s=CFG.s, k=CFG.t, tol=CFG.tol, out=xh.numpy())
    e2e = []
    for _ in range(max(2, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info_e = solver.solve(bh.numpy(), m=CFG.m, s=CFG.s, k=CFG.t, tol=CFG.tol, out=xh.numpy())
        e2e.append(time.perf_counter() - t0)
    assert info_e["status"] == 0

    last = i64[-1]
    launches = sum(i["kernel_launches"] for i in i64) / len(i64)
    k1_ms = sum(i["t_inner_spmv_ms"] for i in ip) / sum(i["n_inner_spmv"] for i in ip)
    hbm, peak_src = _peaks()
    Bn = int(solver.get("block_rows"))  # rows per block in use (the library's choice)
    nblk = -(-n // Bn)
    fused = all(i["n_inner_axpy"] == 0 for i in ip)  # one launch per inner step
    if fused:
        kname = ("k_inner_step (one inner step per launch: fused SpMV + window dots + sketch partials, grid-wide "
                 "arrival, truncated-Arnoldi update; FP64)")
        abytes = alg_bytes_inner_step(n, nnz, CFG.t, 8)
        tkey = "inner_step_fp64_cd3d_128"
    else:
        kname = "k_inner_spmv (fused SpMV + truncated-Arnoldi dots + sketch partials, FP64)"
        abytes = alg_bytes_inner_spmv(n, nnz, CFG.t, CFG.zeta, CFG.s, nblk, 8)
        tkey = "inner_spmv_fp64_cd3d_128"
    n_span = sum(i["n_step_span"] for i in isp)
    span_ms = sum(i["t_step_span_ms"] for i in isp) / n_span if n_span else None
    # the kernel's average launch duration: from the cycle spans (no event between two launches; the gaps between
    # launches count as kernel time) where the step runs as one launch, else from events around every launch
    avg_ms = span_ms if span_ms is not None else k1_ms
    achieved = abytes / (avg_ms / 1e3) / 1e9
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            traffic = json.load(f).get(tkey)
    except Exception:
        pass

    solver.close()
    batch = None if args.no_batch else run_batch(args, dev, stream)
    others = None if args.no_others else run_others(args, dev, stream)
    sweep = None if args.no_others else run_truncation(args, dev, stream)
    ilu = None if args.no_others else run_precond(args, dev, stream)
    cpu = cpu_baseline() if (rank == 0 and not args.no_cpu) else None
    if rank == 0:
        res = {
            "metric": METRIC, "value": sec, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "nnz": nnz, "parallelism": "replicas" if world > 1 else "1gpu",
                       "l2": "inputs larger than L2 (A is 183 MB) and a 256 MB buffer written between steps"},
            "solve": {"outer_iters": last["outer_iters"], "total_inner": last["total_inner"],
                      "rel_res_true": last["rel_res_true"], "inner_k": last["inner_k"],
                      "solves_per_s": 1.0 / sec},
            "variants": {
                "fp32_inner": {"value": statistics.mean(t32), "unit": "s", "outer_iters": i32[-1]["outer_iters"],
                               "total_inner": i32[-1]["total_inner"], "rel_res_true": i32[-1]["rel_res_true"]},
                "bf16_basis": {"value": statistics.mean(t16), "unit": "s", "outer_iters": i16[-1]["outer_iters"],
                               "total_inner": i16[-1]["total_inner"], "rel_res_true": i16[-1]["rel_res_true"]},
            },
            "roofline": {"kernel": kname,
                         "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_source": peak_src, "traffic": traffic,
                         "alg_bytes_per_launch": abytes, "avg_launch_ms": avg_ms,
                         "timing": ("CUDA events on the step stream around each full inner cycle's chain of m step "
                                    "launches (nothing recorded between launches); span / m, the gaps between "
                                    "launches included" if span_ms is not None else
                                    "CUDA events on the step stream around every launch"),
                         "launches_timed": int(n_span if span_ms is not None else sum(i["n_inner_spmv"] for i in ip)),
                         "profiled_solve_s": statistics.mean(ts if span_ms is not None else tp),
                         "per_launch_events": {
                             "avg_launch_ms": k1_ms, "achieved": abytes / (k1_ms / 1e3) / 1e9,
                             "frac": abytes / (k1_ms / 1e3) / 1e9 / hbm,
                             "launches_timed": int(sum(i["n_inner_spmv"] for i in ip)),
                             "profiled_solve_s": statistics.mean(tp),
                             "how": "a pair of events around every launch (the events' own cost included)"}},
            "e2e": {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": 8 * n},
            "batch": batch,
            "workloads": others,
            "truncation_sweep": sweep,
            "precond_ilu0": ilu,
            "gpu_launches": int(round(launches)) * args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(res))
    if dist is not None:
        dist.destroy_process_group()


def _event_time(fn, stream, K, W):
    import torch

    for _ in range(W):
        fn()
    ts, out = [], None
    for _ in range(K):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return statistics.median(ts), out


def run_others(args, dev, stream):
    """The other workloads, each timed with CUDA events on the solver's stream (median of K after W warm-ups):
    2D 64^2 (latency bound: microseconds per solve and solves per second), the random Zipf matrix (FP64, FP32
    inner, BF16 basis), and the differentiation workload (3D 64^3, 16 right-hand sides: forward solves plus the
    adjoint backward through torch.autograd)."""
    import torch

    from paper_2506_18408_gb300 import Solver, sfgmres_solve_autograd

    out = {}
    cfg = workloads.CONFIGS["cd2d_64"]
    A = cfg.build_matrix()
    bd = torch.from_numpy(cfg.build_rhs(A.n)).to(dev)
    sv = Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=cfg.sketch_seed, max_outer=cfg.max_outer,
                stream=stream.cuda_stream)
    for prec in ("fp64", "fp32"):
        sv.set("precision", prec)
        sec, (_, info) = _event_time(lambda: sv.solve(bd, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol), stream, 20, 5)
        out[f"cd2d_64_{prec}"] = {"us_per_solve": sec * 1e6, "solves_per_s": 1.0 / sec,
                                  "outer_iters": info["outer_iters"], "total_inner": info["total_inner"],
                                  "rel_res_true": info["rel_res_true"], "kernel_launches": info["kernel_launches"]}
    sv.close()
    cfg = workloads.CONFIGS["zipf_2m"]
    A = cfg.build_matrix()
    bd = torch.from_numpy(cfg.build_rhs(A.n)).to(dev)
    sv = Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=cfg.sketch_seed, max_outer=cfg.max_outer,
                stream=stream.cuda_stream)
    for prec in ("fp64", "fp32", "bf16"):
        sv.set("precision", prec)
        sec, (_, info) = _event_time(lambda: sv.solve(bd, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol), stream, 3, 1)
        out[f"zipf_2m_{prec}"] = {"s_per_solve": sec, "outer_iters": info["outer_iters"],
                                  "total_inner": info["total_inner"], "rel_res_true": info["rel_res_true"],
                                  "nnz": int(A.nnz)}
    sv.close()
    cfg = workloads.CONFIGS["cd3d_64"]
    A = cfg.build_matrix()
    B = torch.from_numpy(workloads.rhs(A.n, seed=0, nrhs=16)).to(dev)
    xs = torch.from_numpy(workloads.rhs(A.n, seed=0, stream=workloads.STREAM_XSTAR, nrhs=16)).to(dev)
    vals = torch.from_numpy(A.val).to(dev)
    sv = Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=cfg.sketch_seed, max_outer=cfg.max_outer,
                stream=stream.cuda_stream)

    def fwd_bwd():
        v = vals.clone().requires_grad_(True)
        b = B.clone().requires_grad_(True)
        x = sfgmres_solve_autograd(sv, v, b, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol)
        loss = ((x - xs) ** 2).sum()
        loss.backward()
        return loss

    for prec in ("fp64", "fp32"):
        sv.set("precision", prec)
        sec, _ = _event_time(fwd_bwd, stream, 3, 1)
        out[f"cd3d_64_x16_grad_{prec}"] = {"s_forward_backward": sec, "rhs": 16}
    # the 16 right-hand sides as one batched FP32-inner solve against 16 plain FP64 solves one after another
    Bf = B.reshape(-1).contiguous()
    kw = dict(m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol)
    sv.set("precision", "fp32")
    t_batch, _ = _event_time(lambda: sv.solve_batch(Bf, nrhs=16, **kw), stream, 3, 1)
    sv.set("precision", "fp64")

    def sequential():
        for r in range(16):
            sv.solve(B[r], **kw)

    t_seq, _ = _event_time(sequential, stream, 2, 1)
    out["cd3d_64_x16_batched_vs_plain"] = {"batched_fp32_inner_s": t_batch, "plain_fp64_sequential_s": t_seq,
                                           "speedup": t_seq / t_batch}
    sv.close()
    return out


def run_truncation(args, dev, stream):
    """The paper's preferred setting (Section 4.1) on the 128^3 workload: a Clarkson-Woodruff sketch (zeta = 1),
    s = 2 k_max = 1000, k_max = m = 500, rules C1-C3 with the condition threshold 1e15, truncation t = 0..5; time to
    1e-8 (median of 2 after 1 warm-up, CUDA events), outer and inner counts, and for t = 2 a profiled solve giving the
    per-launch time of the inner kernel and of the sketched-QR update at this sketch size."""
    import torch

    from paper_2506_18408_gb300 import Solver

    A = CFG.build_matrix()
    bd = torch.from_numpy(CFG.build_rhs(A.n)).to(dev)
    m, s = 500, 1000
    sv = Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=CFG.sketch_seed, zeta=1, max_outer=CFG.max_outer,
                stream=stream.cuda_stream)
    out = {"workload": "cd3d_128 with a Clarkson-Woodruff sketch (zeta=1), s=1000, m=k_max=500, C1-C3, tol 1e-8",
           "per_t": {}}
    for t in range(6):
        sec, (_, info) = _event_time(lambda: sv.solve(bd, m=m, s=s, k=t, tol=CFG.tol), stream, 2, 1)
        ks = info["inner_k"]
        out["per_t"][str(t)] = {"s_per_solve": sec, "outer_iters": info["outer_iters"],
                                "total_inner": info["total_inner"], "inner_k_min": min(ks), "inner_k_max": max(ks),
                                "inner_reasons": sorted(set(info["inner_reason"])),
                                "rel_res_true": info["rel_res_true"]}
    sv.set("profile", 1)
    _, info = sv.solve(bd, m=m, s=s, k=2, tol=CFG.tol)
    sv.set("profile", 0)
    out["t2_profile"] = {"inner_step_us": 1e3 * info["t_inner_spmv_ms"] / max(1, info["n_inner_spmv"]),
                         "qr_update_us": 1e3 * info["t_qr_ms"] / max(1, info["n_qr"]),
                         "qr_updates": info["n_qr"], "inner_steps": info["n_inner_spmv"]}
    sv.close()
    return out


def run_precond(args, dev, stream):
    """ILU(0) right preconditioning in a multicolour order (Section 4's "-p" runs) on the 128^3 workload: time to 1e-8
    (median of 3 after 1 warm-up, CUDA events), outer and inner counts, against the unpreconditioned FP64 solve on the
    same handle and inputs."""
    import torch

    from paper_2506_18408_gb300 import Solver

    A = CFG.build_matrix()
    bd = torch.from_numpy(CFG.build_rhs(A.n)).to(dev)
    sv = Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=CFG.sketch_seed, max_outer=CFG.max_outer,
                stream=stream.cuda_stream)
    out = {"workload": WORKLOAD + "; ILU(0) of the red-black ordered matrix as right preconditioner"}
    for pc in (0, 1):
        sv.set("precond", pc)
        sec, (_, info) = _event_time(lambda: sv.solve(bd, m=CFG.m, s=CFG.s, k=CFG.t, tol=CFG.tol), stream, 3, 1)
        out["ilu0" if pc else "none"] = {"s_per_solve": sec, "outer_iters": info["outer_iters"],
                                         "total_inner": info["total_inner"], "rel_res_true": info["rel_res_true"]}
    out["colours"] = sv.precond_info()[1]
    sv.close()
    return out


def run_batch(args, dev, stream):
    """The batched form: 512 2D convection-diffusion systems x 4 right-hand sides (2048 problems, 176.6M unknowns)
    in one lockstep solve, FP32 inner cycles with the FP64 outer FGMRES; reported as solves per second."""
    import torch

    from paper_2506_18408_gb300 import Solver

    cfg = workloads.CONFIGS["batch_512"]
    A = cfg.build_matrix()
    b = cfg.build_rhs(A.n)
    sv = Solver(list(A.sys_n), A.row_ptr, A.col, A.val, sketch_seed=cfg.sketch_seed, zeta=cfg.zeta,
                max_outer=cfg.max_outer, precision=cfg.precision, stream=stream.cuda_stream)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.empty_like(bd)
    del b
    P = len(A.sys_n) * cfg.nrhs
    t0 = time.perf_counter()
    tile = sv.autotune(nrhs=cfg.nrhs, m=cfg.m, s=cfg.s, k=cfg.t)  # row-block size and SpMV width, outside the timing
    tune_s = time.perf_counter() - t0
    kw = dict(nrhs=cfg.nrhs, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol, out=xd)
    for _ in range(args.batch_warmup):
        sv.solve_batch(bd, **kw)
    times = []
    for _ in range(args.batch_steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info = sv.solve_batch(bd, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    sv.close()
    sec = statistics.mean(times)
    st = info["status_p"]
    # algorithmic bytes of the whole batch (FP32 inner cycles: FP32 values and basis), problem by problem
    rows_nnz = np.diff(A.row_ptr)
    sys_off = np.concatenate([[0], np.cumsum(A.sys_n)])
    sys_nnz = [int(rows_nnz[sys_off[q]:sys_off[q + 1]].sum()) for q in range(len(A.sys_n))]
    abytes = 0
    for p in range(P):
        q = p // cfg.nrhs
        abytes += alg_bytes_solve(int(A.sys_n[q]), sys_nnz[q], cfg.t, 4, 4, info["inner_steps_p"][p],
                                  info["outer_iters_p"][p])
    hbm, peak_src = _peaks()
    # the plain FP64 solver on the same inputs, problem by problem, on a seeded simple random sample of problems;
    # the batch total is extrapolated from the sample mean, with its standard error (finite-population corrected)
    rng = np.random.default_rng([0, workloads.STREAM_SAMPLE])
    sample = sorted(rng.choice(P, size=min(P, args.batch_sample), replace=False).tolist())
    blocks = workloads.split_blocks(A)
    sl = workloads.problem_slices(A.sys_n, cfg.nrhs)
    t_each = []
    for p in sample:
        q, a0, nq = sl[p]
        Aq = blocks[q]
        one = Solver(Aq.n, Aq.row_ptr, Aq.col, Aq.val, sketch_seed=cfg.sketch_seed, zeta=cfg.zeta,
                     max_outer=cfg.max_outer, stream=stream.cuda_stream)
        bq = bd[a0:a0 + nq].contiguous()
        tq, _ = _event_time(lambda: one.solve(bq, m=cfg.m, s=cfg.s, k=cfg.t, tol=cfg.tol), stream, 1, 1)
        t_each.append(tq)
        one.close()
    t_plain = float(sum(t_each))
    ns = len(t_each)
    plain_est = t_plain * P / ns
    sd = statistics.stdev(t_each) if ns > 1 else 0.0
    plain_se = P * sd / math.sqrt(ns) * math.sqrt(max(0.0, 1.0 - ns / P))
    return {"workload": "batch_512: 512 2D convection-diffusion systems, sides U{32..512}, beta~U(0,50)^2, "
                        "4 RHS ~N(0,1) each; m=40, k=2, s=160, FP32 inner + FP64 outer, tol 1e-8",
            "value": P / sec, "unit": "solves/s", "time_s": sec, "steps": args.batch_steps,
            "warmup": args.batch_warmup, "problems": P, "unknowns": int(A.n) * cfg.nrhs, "nnz": int(A.nnz),
            "converged": int(sum(1 for v in st if v == 0)), "lockstep_outer": info["lockstep_outer"],
            "max_outer": max(info["outer_iters_p"]), "total_inner": info["total_inner"],
            "max_rel_res_true": max(info["rel_res_true_p"]), "kernel_launches": info["kernel_launches"],
            "autotune": {"block_rows": tile[0], "spmv_vector": tile[1], "step_ms": tile[2], "tune_s": tune_s},
            "roofline": {"bound": "hbm", "alg_bytes": abytes, "achieved": abytes / sec / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": abytes / sec / 1e9 / hbm, "peak_source": peak_src,
                         "counted": "per problem: inner steps (A in FP32, basis FP32), z = B y per cycle, outer "
                                    "steps (FP64 SpMV + CGS2)"},
            "plain_fp64_per_problem": {"sample_size": ns, "sample_s": t_plain, "extrapolated_s": plain_est,
                                       "extrapolated_stderr_s": plain_se, "batched_speedup": plain_est / sec,
                                       "batched_speedup_stderr": plain_se / sec}}


def _oracle_outer_iters():
    """Outer FGMRES iterations of the oracle's own 128^3 FP64 solve (tests/golden/oracle_runs.json, written by
    tests/golden/make_oracle_runs.py from the oracle alone): the factor from a one-outer-iteration sample to a solve."""
    with open(os.path.join(ROOT, "tests", "golden", "oracle_runs.json")) as f:
        return int(json.load(f)["cd3d_128_fp64"]["outer_iters"])


def cpu_baseline():
    """The oracle as it stands, one full solve of the same workload to 1e-8 on one host core, timed (about a minute
    on the GPU host's cores)."""
    from oracle import fgmres as ofg
    from oracle import sketch as osk

    A = CFG.build_matrix().to_scipy()
    b = CFG.build_rhs(A.shape[0])
    osk.sketch_matrix(A.shape[0], CFG.s, CFG.zeta, CFG.sketch_seed)  # first construction outside the timing
    t0 = time.perf_counter()
    r = ofg.fgmres(A, b, m=CFG.m, s=CFG.s, t=CFG.t, tol=CFG.tol, max_outer=CFG.max_outer, zeta=CFG.zeta,
                   sketch_seed=CFG.sketch_seed)
    dt = time.perf_counter() - t0
    return {"value": dt, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": f"one full solve to 1e-8 ({r.outer_iters} outer iterations, {sum(r.inner_k)} inner steps, "
                      f"rel. residual {r.rel_res_true:.2e}), timed"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import fgmres as ofg
    from oracle import sketch as osk

    A = CFG.build_matrix().to_scipy()
    b = CFG.build_rhs(A.shape[0])
    osk.sketch_matrix(A.shape[0], CFG.s, CFG.zeta, CFG.sketch_seed)
    # a step = one bounded sample: the first outer FGMRES iteration (a full inner cycle of m = 100 sGMRES steps plus
    # the outer step), scaled by the oracle's own outer iteration count for this solve (stored with its other runs)
    J = _oracle_outer_iters()
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ofg.fgmres(A, b, m=CFG.m, s=CFG.s, t=CFG.t, tol=CFG.tol, max_outer=1, zeta=CFG.zeta,
                   sketch_seed=CFG.sketch_seed)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt * J)
    v = statistics.mean(times)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": f"1 outer iteration ({CFG.m} inner steps + outer step) per timed step, x "
                                   f"{J} outer iterations of the oracle's solve"},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile-case", nargs="?", const="cd3d_128", default=None,
                    help="short solves for ncu captures: cd3d_128 (default), zipf_2m, qr_cd3d (one inner cycle "
                         "of m = 100), or cd2d_64 (two full solves of the small 2D workload)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-solve line")
    ap.add_argument("--no-others", action="store_true", help="skip the other workloads' lines")
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--batch-warmup", type=int, default=1)
    ap.add_argument("--batch-sample", type=int, default=64,
                    help="problems solved one by one with the plain FP64 solver for the batch's baseline")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
