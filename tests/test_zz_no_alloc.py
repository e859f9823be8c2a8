"""The allocation-free sketch entry point (for callers that cannot call cudaMalloc) against the handle's sketch.

sfgmres_sketch_apply_noalloc keeps its scratch in a static device array shared by all calls; calls in a row, with
different sizes and inputs (the last at the largest sketch, s = 4096, whose block accumulators need more than the
default 48 KiB of shared memory), must each agree with sfgmres_sketch_apply (which builds gather lists in memory a
solver handle allocates) to the 1e-13 relative tolerance the other sketch tests use.  This file is collected last.
"""
import numpy as np
import pytest

import workloads
from gpu_common import dev_vec, need_gpu, rel_err, torch

pytestmark = pytest.mark.gpu


def test_noalloc_sketch_matches_handle_sketch_in_a_row():
    need_gpu()
    from paper_2506_18408_gb300 import Solver
    from paper_2506_18408_gb300 import sfgmres as py

    stream = torch.cuda.current_stream().cuda_stream
    cases = [(70_001, 400, 8, 5, 11), (2_097_152, 240, 8, 1, 12), (50_000, 4096, 8, 3, 13)]  # (n, s, zeta, seeds)
    for n, s, zeta, seed, rseed in cases:
        A = workloads.convdiff(n, (1.0,))  # only n matters for the sketch
        sv = Solver(A.n, A.row_ptr, A.col, A.val, sketch_seed=seed, zeta=zeta)
        v = dev_vec(workloads.rhs(n, seed=rseed))
        ref = sv.sketch(v, s).cpu().numpy()
        c = torch.full((s,), float("nan"), dtype=torch.float64, device="cuda")
        py.sfgmres_sketch_apply_noalloc(n, s, zeta, seed, v, c, stream)
        torch.cuda.synchronize()
        got = c.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_err(got, ref) <= 1e-13, (n, s, rel_err(got, ref))
        sv.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    need_gpu()
    from paper_2506_18408_gb300 import sfgmres as py

    v = torch.zeros(16, dtype=torch.float64, device="cuda")
    c = torch.zeros(8, dtype=torch.float64, device="cuda")
    for args in ((16, 5000, 8), (16, 4, 8), (2**31 - 1, 4096, 8)):
        with pytest.raises(py.SFGMRESError) as e:
            py.sfgmres_sketch_apply_noalloc(args[0], args[1], args[2], 1, v, c)
        assert e.value.code == py.ERR_INVALID_ARG
        assert "sfgmres_sketch_apply_noalloc" in str(e.value)
