"""Write tests/golden/oracle_runs.json: the oracle's full FGMRES-sGMRES solves of the full-size workloads, scalars only.

The GPU parity tests compare the CUDA solver's outer iteration counts, per-step residual estimates, inner lengths and
Eq. 5 quantities with these runs.  Full oracle solves at n = 2M take minutes each on one core, so they are computed
once here, on the CPU, from the same seeded inputs the tests regenerate (NumPy's PCG64 streams are the same on every
platform), and stored.  Only ``oracle/`` and the input generators of ``workloads`` are called; nothing here touches
the CUDA path.

    python tests/golden/make_oracle_runs.py [name ...]      # default: every run below; about 20 minutes in total
"""
from __future__ import annotations

import json
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
OUT = os.path.join(HERE, "oracle_runs.json")

# (workload config, inner precision of the sGMRES cycles)
RUNS = {
    "cd3d_128_fp64": ("cd3d_128", "fp64"),
    "cd3d_128_fp32": ("cd3d_128", "fp32"),
    "cd3d_128_bf16": ("cd3d_128", "bf16"),
    "zipf_2m_fp64": ("zipf_2m", "fp64"),
    "zipf_2m_fp32": ("zipf_2m", "fp32"),
}


def run(name: str) -> dict:
    import workloads
    from oracle import fgmres as ofg

    cfg_name, inner = RUNS[name]
    cfg = workloads.CONFIGS[cfg_name]
    A = cfg.build_matrix()
    b = cfg.build_rhs(A.n)
    t0 = time.time()
    r = ofg.fgmres(A.to_scipy(), b, m=cfg.m, s=cfg.s, t=cfg.t, tol=cfg.tol, max_outer=cfg.max_outer,
                   sketch_seed=cfg.sketch_seed, zeta=cfg.zeta, inner=inner, trace=True)
    return {"workload": cfg_name, "inner": inner, "m": cfg.m, "s": cfg.s, "t": cfg.t, "tol": cfg.tol,
            "max_outer": cfg.max_outer, "n": int(A.n), "nnz": int(A.nnz), "status": int(r.status),
            "outer_iters": int(r.outer_iters), "rel_res_true": float(r.rel_res_true),
            "est_hist": [float(v) for v in r.est_hist], "ffom_hist": [float(v) for v in r.ffom_hist],
            "inner_k": [int(v) for v in r.inner_k], "inner_reason": [int(v) for v in r.inner_reason],
            "rhat_hist": [float(v) for v in r.rhat_hist], "rho_hist": [float(v) for v in r.rho_hist],
            "oracle_seconds": round(time.time() - t0, 1)}


def main(names):
    old = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            old = json.load(f)
    with ProcessPoolExecutor(max_workers=min(len(names), 4), mp_context=mp.get_context("spawn")) as ex:
        for name, res in zip(names, ex.map(run, names)):
            old[name] = res
            print(name, res["outer_iters"], res["inner_k"], res["oracle_seconds"], flush=True)
    with open(OUT, "w") as f:
        json.dump(dict(sorted(old.items())), f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or list(RUNS))
