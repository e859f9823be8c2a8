"""Thin ctypes binding of the sketched-FGMRES C ABI (``include/sfgmres.h``).

Only argument marshalling happens here: every step of a solve runs in the CUDA library ``_lib/libsfgmres.so``.
PyTorch supplies device memory and the current CUDA stream; NumPy arrays are accepted as host buffers.  If the
library has not been built the functions raise ``RuntimeError`` -- there is no CPU fallback.

The functions named ``sfgmres_*`` mirror the C entry points one to one; :class:`Solver` wraps a handle for
convenience.  Parameter names follow the paper through this mapping: ``m`` = maximum inner sGMRES basis size (the
paper's k_max, rule C1), ``k`` = Arnoldi truncation depth (the paper's t), ``s`` = sketch rows.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsfgmres.so")

OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2
ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NAN = -1, -2, -3, -4
CSR_HOST = 1
OPT_PRECISION, OPT_ZETA, OPT_COND_THRESHOLD, OPT_C3, OPT_MAX_OUTER, OPT_SKETCH_KIND, OPT_PROFILE, \
    OPT_SPMV_VECTOR, OPT_BLOCK_ROWS, OPT_GRAPH = range(1, 11)
OPT_FUSED_STEP, OPT_STEP_WAIT_EXTRA, OPT_OUTER_VARIANT, OPT_PRECOND = range(13, 17)
SOLVE_TRANSPOSE = 1
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2}
SKETCH_KIND = {"sparse_sign": 0, "identity": 1}

EXPORTED = ["sfgmres_create", "sfgmres_create_batch", "sfgmres_set_option", "sfgmres_get_option", "sfgmres_solve",
            "sfgmres_solve_transpose", "sfgmres_solve_batch", "sfgmres_solve_restarted", "sfgmres_solve_multilevel", "sfgmres_precond_info",
            "sfgmres_autotune", "sfgmres_update_values", "sfgmres_pattern_outer", "sfgmres_inner_cycle",
            "sfgmres_sketch_apply", "sfgmres_sketch_apply_noalloc", "sfgmres_sketch_pattern", "sfgmres_spmv",
            "sfgmres_destroy", "sfgmres_last_error", "sfgmres_version"]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("outer_iters", C.c_int32), ("total_inner", C.c_int32),
                ("hist_cap", C.c_int32), ("inner_k", C.POINTER(C.c_int32)), ("inner_reason", C.POINTER(C.c_int32)),
                ("res_est", C.POINTER(C.c_double)), ("ffom_res", C.POINTER(C.c_double)),
                ("rel_res_true", C.c_double), ("rel_res_est", C.c_double), ("kernel_launches", C.c_int64),
                ("t_inner_spmv_ms", C.c_double), ("n_inner_spmv", C.c_int64), ("t_inner_axpy_ms", C.c_double),
                ("n_inner_axpy", C.c_int64), ("t_qr_ms", C.c_double), ("n_qr", C.c_int64),
                ("t_total_ms", C.c_double), ("inner_res", C.POINTER(C.c_double)),
                ("inner_rho", C.POINTER(C.c_double)), ("t_step_span_ms", C.c_double),
                ("n_step_span", C.c_int64)]


class BatchStats(C.Structure):
    _fields_ = [("problems", C.c_int32), ("lockstep_outer", C.c_int32), ("total_inner", C.c_int64),
                ("status", C.POINTER(C.c_int32)), ("outer_iters", C.POINTER(C.c_int32)),
                ("rel_res_true", C.POINTER(C.c_double)), ("rel_res_est", C.POINTER(C.c_double)),
                ("kernel_launches", C.c_int64), ("t_total_ms", C.c_double), ("inner_steps", C.POINTER(C.c_int32))]


_lib = None


def load():
    """Load the CUDA library (once); raises RuntimeError when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run __graft_entry__.build() first")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, f64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint64
    lib.sfgmres_create.argtypes = [C.POINTER(vp), i64, i64, vp, vp, vp, u64, i32, vp]
    lib.sfgmres_create_batch.argtypes = [C.POINTER(vp), i32, vp, i64, vp, vp, vp, u64, i32, vp]
    lib.sfgmres_set_option.argtypes = [vp, i32, f64]
    lib.sfgmres_get_option.argtypes = [vp, i32, C.POINTER(f64)]
    lib.sfgmres_solve.argtypes = [vp, vp, vp, vp, i32, i32, i32, f64, C.POINTER(Stats)]
    lib.sfgmres_solve_transpose.argtypes = [vp, vp, vp, vp, i32, i32, i32, f64, C.POINTER(Stats)]
    lib.sfgmres_solve_batch.argtypes = [vp, i32, vp, vp, vp, i32, i32, i32, f64, i32, C.POINTER(BatchStats)]
    lib.sfgmres_autotune.argtypes = [vp, i32, i32, i32, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(f64)]
    lib.sfgmres_solve_restarted.argtypes = [vp, vp, vp, vp, i32, i32, i32, f64, i32, vp, C.POINTER(i32)]
    lib.sfgmres_solve_multilevel.argtypes = [vp, vp, vp, vp, i32, i32, i32, f64, i32, vp, C.POINTER(Stats)]
    lib.sfgmres_precond_info.argtypes = [vp, vp, C.POINTER(i32), vp]
    lib.sfgmres_update_values.argtypes = [vp, vp]
    lib.sfgmres_pattern_outer.argtypes = [vp, vp, vp, f64, vp]
    lib.sfgmres_inner_cycle.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, C.POINTER(i32), C.POINTER(i32)]
    lib.sfgmres_sketch_apply.argtypes = [vp, i32, vp, vp]
    lib.sfgmres_sketch_apply_noalloc.argtypes = [i64, i32, i32, u64, vp, vp, vp]
    lib.sfgmres_sketch_pattern.argtypes = [vp, i32, vp, vp]
    lib.sfgmres_spmv.argtypes = [vp, vp, vp]
    lib.sfgmres_destroy.argtypes = [vp]
    lib.sfgmres_last_error.argtypes = [vp]
    lib.sfgmres_last_error.restype = C.c_char_p
    lib.sfgmres_version.argtypes = []
    lib.sfgmres_version.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("sfgmres_last_error", "sfgmres_version"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class SFGMRESError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sfgmres error {code}: {msg}")
        self.code = code


def _ptr(a) -> Optional[int]:
    """Address of a torch tensor or numpy array (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported buffer type {type(a)}")


def _check(h, rc: int, allow_positive: bool = True) -> int:
    if rc < 0 or (rc > 0 and not allow_positive):
        raise SFGMRESError(rc, load().sfgmres_last_error(h).decode())
    return rc


# ---- one-to-one wrappers of the C entry points -------------------------------------------------------------------
def sfgmres_version() -> str:
    return load().sfgmres_version().decode()


def sfgmres_create(n: int, nnz: int, row_ptr, col_idx, vals, sketch_seed: int, flags: int = 0,
                   stream: Optional[int] = None) -> int:
    lib = load()
    h = C.c_void_p()
    rc = lib.sfgmres_create(C.byref(h), n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), sketch_seed, flags,
                            stream)
    if rc != 0:
        raise SFGMRESError(rc, lib.sfgmres_last_error(None).decode())
    return h.value


def sfgmres_create_batch(sys_n, nnz: int, row_ptr, col_idx, vals, sketch_seed: int, flags: int = 0,
                         stream: Optional[int] = None) -> int:
    lib = load()
    sn = np.ascontiguousarray(sys_n, dtype=np.int64)
    h = C.c_void_p()
    rc = lib.sfgmres_create_batch(C.byref(h), len(sn), _ptr(sn), nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(vals),
                                  sketch_seed, flags, stream)
    if rc != 0:
        raise SFGMRESError(rc, lib.sfgmres_last_error(None).decode())
    return h.value


def sfgmres_set_option(h: int, key: int, value: float) -> None:
    _check(h, load().sfgmres_set_option(h, key, float(value)))


def sfgmres_get_option(h: int, key: int) -> float:
    v = C.c_double()
    _check(h, load().sfgmres_get_option(h, key, C.byref(v)))
    return v.value


def sfgmres_solve(h: int, b, x0, x, m: int, s: int, k: int, tol: float, stats: Optional[Stats] = None) -> int:
    return _check(h, load().sfgmres_solve(h, _ptr(b), _ptr(x0), _ptr(x), m, s, k, tol,
                                          C.byref(stats) if stats is not None else None))


def sfgmres_solve_transpose(h: int, b, x0, x, m: int, s: int, k: int, tol: float,
                            stats: Optional[Stats] = None) -> int:
    return _check(h, load().sfgmres_solve_transpose(h, _ptr(b), _ptr(x0), _ptr(x), m, s, k, tol,
                                                    C.byref(stats) if stats is not None else None))


def sfgmres_solve_batch(h: int, nrhs: int, b, x0, x, m: int, s: int, k: int, tol: float, flags: int = 0,
                        stats: Optional[BatchStats] = None) -> int:
    return _check(h, load().sfgmres_solve_batch(h, nrhs, _ptr(b), _ptr(x0), _ptr(x), m, s, k, tol, flags,
                                                C.byref(stats) if stats is not None else None))


def sfgmres_autotune(h: int, nrhs: int, m: int, s: int, k: int):
    """Time candidate row-block sizes / SpMV widths and keep the fastest; returns (block_rows, spmv_vector, step_ms)."""
    b, v, t = C.c_int32(), C.c_int32(), C.c_double()
    _check(h, load().sfgmres_autotune(h, nrhs, m, s, k, C.byref(b), C.byref(v), C.byref(t)), allow_positive=False)
    return b.value, v.value, t.value


def sfgmres_update_values(h: int, vals) -> None:
    _check(h, load().sfgmres_update_values(h, _ptr(vals)), allow_positive=False)


def sfgmres_pattern_outer(h: int, u, v, alpha: float, out) -> None:
    _check(h, load().sfgmres_pattern_outer(h, _ptr(u), _ptr(v), float(alpha), _ptr(out)), allow_positive=False)


def sfgmres_solve_restarted(h: int, b, x0, x, m: int, s: int, k: int, tol: float, max_cycles: int,
                            res_hist=None) -> tuple:
    """Returns ``(status, cycles)``; ``res_hist`` (NumPy float64[max_cycles + 1]) receives ||r_c|| / ||b||."""
    cyc = C.c_int32()
    rc = _check(h, load().sfgmres_solve_restarted(h, _ptr(b), _ptr(x0), _ptr(x), m, s, k, tol, max_cycles,
                                                  _ptr(res_hist), C.byref(cyc)))
    return rc, cyc.value


def sfgmres_solve_multilevel(h: int, b, x0, x, m: int, s: int, k: int, tol: float, level_steps,
                             stats: Optional[Stats] = None) -> int:
    """Multi-level FGMRES: ``level_steps`` lists the outer-step budgets of the FGMRES levels below the top."""
    ls = np.ascontiguousarray(level_steps, dtype=np.int32)
    return _check(h, load().sfgmres_solve_multilevel(h, _ptr(b), _ptr(x0), _ptr(x), m, s, k, tol, len(ls), _ptr(ls),
                                                     C.byref(stats) if stats is not None else None))


def sfgmres_precond_info(h: int, colour=None, lu=None) -> int:
    """The ILU(0) preconditioner's colouring (int32[n]) and factor values in A's entry order (float64[nnz]), both
    NumPy arrays filled in place (either may be None); returns the number of colours."""
    nc = C.c_int32()
    _check(h, load().sfgmres_precond_info(h, _ptr(colour), C.byref(nc), _ptr(lu)), allow_positive=False)
    return nc.value


def sfgmres_inner_cycle(h: int, v, z, m: int, s: int, k: int, basis=None, y=None):
    kk, rr = C.c_int32(), C.c_int32()
    rc = _check(h, load().sfgmres_inner_cycle(h, _ptr(v), _ptr(z), m, s, k, _ptr(basis), _ptr(y), C.byref(kk),
                                              C.byref(rr)))
    return rc, kk.value, rr.value


def sfgmres_sketch_apply(h: int, s: int, v, c) -> None:
    _check(h, load().sfgmres_sketch_apply(h, s, _ptr(v), _ptr(c)), allow_positive=False)


def sfgmres_sketch_apply_noalloc(n: int, s: int, zeta: int, sketch_seed: int, v, c, stream=None) -> None:
    """c = S v with no device allocation (for callers that cannot allocate); enqueued on ``stream``."""
    lib = load()
    rc = lib.sfgmres_sketch_apply_noalloc(n, s, zeta, sketch_seed, _ptr(v), _ptr(c), stream)
    if rc != 0:
        raise SFGMRESError(rc, lib.sfgmres_last_error(None).decode())


def sfgmres_sketch_pattern(h: int, s: int, rows, signs) -> None:
    _check(h, load().sfgmres_sketch_pattern(h, s, _ptr(rows), _ptr(signs)), allow_positive=False)


def sfgmres_spmv(h: int, x, y) -> None:
    _check(h, load().sfgmres_spmv(h, _ptr(x), _ptr(y)), allow_positive=False)


def sfgmres_destroy(h: int) -> None:
    load().sfgmres_destroy(h)


def sfgmres_last_error(h: Optional[int]) -> str:
    return load().sfgmres_last_error(h).decode()


# ---- convenience wrapper -------------------------------------------------------------------------------------------
class Solver:
    """A solver handle for one CSR matrix, or for a batch of systems given as one block-diagonal CSR matrix (``n`` a
    list of the systems' orders; see ``sfgmres_create_batch``).

    ``row_ptr``/``col``/``val`` may be NumPy arrays (host; copied by the library) or CUDA tensors (int64, int32,
    float64).  ``options`` are set through :meth:`set` (``precision`` in {"fp64","fp32","bf16"}, ``zeta``,
    ``cond_threshold``, ``c3``, ``max_outer``, ``sketch_kind`` in {"sparse_sign","identity"}, ``profile`` (0; 1 =
    events around every kernel launch, reported as ``t_inner_spmv_ms`` etc.; 2 = events around each full inner
    cycle's chain of step launches, reported as ``t_step_span_ms`` / ``n_step_span``),
    ``spmv_vector``).
    """

    _KEYS = {"precision": OPT_PRECISION, "zeta": OPT_ZETA, "cond_threshold": OPT_COND_THRESHOLD, "c3": OPT_C3,
             "max_outer": OPT_MAX_OUTER, "sketch_kind": OPT_SKETCH_KIND, "profile": OPT_PROFILE,
             "spmv_vector": OPT_SPMV_VECTOR, "block_rows": OPT_BLOCK_ROWS, "graph": OPT_GRAPH,
             "fused_step": OPT_FUSED_STEP, "step_wait_extra": OPT_STEP_WAIT_EXTRA,
             "outer_variant": OPT_OUTER_VARIANT, "precond": OPT_PRECOND}

    def __init__(self, n, row_ptr, col, val, sketch_seed: int = 1, stream=None, **options):
        import torch

        sys_n = [int(v) for v in np.atleast_1d(np.asarray(n))]
        self.sys_n = sys_n
        self.nsys = len(sys_n)
        self.n = int(sum(sys_n))
        host = isinstance(row_ptr, np.ndarray)
        if host:
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            val = np.ascontiguousarray(val, dtype=np.float64)
        nnz = int(row_ptr[-1])
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        if self.nsys == 1:
            self.h = sfgmres_create(self.n, nnz, row_ptr, col, val, sketch_seed, CSR_HOST if host else 0, stream)
        else:
            self.h = sfgmres_create_batch(sys_n, nnz, row_ptr, col, val, sketch_seed, CSR_HOST if host else 0,
                                          stream)
        self.nnz = nnz
        for key, v in options.items():
            self.set(key, v)

    def set(self, key: str, value) -> None:
        if key == "precision" and isinstance(value, str):
            value = PRECISION[value]
        if key == "sketch_kind" and isinstance(value, str):
            value = SKETCH_KIND[value]
        sfgmres_set_option(self.h, self._KEYS[key], float(value))

    def get(self, key: str) -> float:
        return sfgmres_get_option(self.h, self._KEYS[key])

    def solve(self, b, x0=None, *, m: int, s: int, k: int, tol: float = 1e-8, out=None, hist_cap: int = 1000,
              transpose: bool = False, level_steps=None):
        """Solve ``A x = b`` (``A^T x = b`` with ``transpose``); ``b``/``x0``/``out`` are float64 CUDA tensors or NumPy
        arrays.  ``level_steps`` (a list of outer-step budgets) runs the multi-level FGMRES with that many levels
        below the top (``sfgmres_solve_multilevel``).  Returns ``(x, info)``."""
        import torch

        if out is None:
            out = torch.empty_like(b) if hasattr(b, "data_ptr") else np.empty_like(b)
        st = Stats()
        kh = (C.c_int32 * hist_cap)()
        rh = (C.c_int32 * hist_cap)()
        eh = (C.c_double * hist_cap)()
        fh = (C.c_double * hist_cap)()
        ih = (C.c_double * hist_cap)()
        qh = (C.c_double * hist_cap)()
        st.hist_cap = hist_cap
        st.inner_res = C.cast(ih, C.POINTER(C.c_double))
        st.inner_rho = C.cast(qh, C.POINTER(C.c_double))
        st.inner_k = C.cast(kh, C.POINTER(C.c_int32))
        st.inner_reason = C.cast(rh, C.POINTER(C.c_int32))
        st.res_est = C.cast(eh, C.POINTER(C.c_double))
        st.ffom_res = C.cast(fh, C.POINTER(C.c_double))
        if level_steps is None:
            rc = (sfgmres_solve_transpose if transpose else sfgmres_solve)(self.h, b, x0, out, m, s, k, tol, st)
        else:
            rc = sfgmres_solve_multilevel(self.h, b, x0, out, m, s, k, tol, level_steps, st)
        J = st.outer_iters
        cnt = min(J + (1 if rc == BREAKDOWN else 0), hist_cap)
        info = {"status": rc, "outer_iters": J, "total_inner": st.total_inner, "rel_res_true": st.rel_res_true,
                "rel_res_est": st.rel_res_est, "inner_k": list(kh[:cnt]), "inner_reason": list(rh[:cnt]),
                "res_est": list(eh[: min(J, hist_cap)]), "ffom_res": list(fh[: min(J, hist_cap)]),
                "inner_res": list(ih[: min(J, hist_cap)]), "inner_rho": list(qh[: min(J, hist_cap)]),
                "kernel_launches": st.kernel_launches, "t_total_ms": st.t_total_ms,
                "t_inner_spmv_ms": st.t_inner_spmv_ms, "n_inner_spmv": st.n_inner_spmv,
                "t_inner_axpy_ms": st.t_inner_axpy_ms, "n_inner_axpy": st.n_inner_axpy, "t_qr_ms": st.t_qr_ms,
                "n_qr": st.n_qr, "t_step_span_ms": st.t_step_span_ms, "n_step_span": st.n_step_span}
        return out, info

    def solve_batch(self, b, x0=None, *, nrhs: int, m: int, s: int, k: int, tol: float = 1e-8, out=None,
                    transpose: bool = False):
        """Solve for ``nrhs`` right-hand sides per system at once; ``b``/``x0``/``out`` hold ``nrhs * n`` values in
        problem order (system-major, then right-hand side).  Returns ``(x, info)`` with per-problem lists."""
        import torch

        if out is None:
            out = torch.empty_like(b) if hasattr(b, "data_ptr") else np.empty_like(b)
        P = self.nsys * nrhs
        st = BatchStats()
        sa = (C.c_int32 * P)()
        oa = (C.c_int32 * P)()
        ra = (C.c_double * P)()
        ea = (C.c_double * P)()
        ka = (C.c_int32 * P)()
        st.inner_steps = C.cast(ka, C.POINTER(C.c_int32))
        st.status = C.cast(sa, C.POINTER(C.c_int32))
        st.outer_iters = C.cast(oa, C.POINTER(C.c_int32))
        st.rel_res_true = C.cast(ra, C.POINTER(C.c_double))
        st.rel_res_est = C.cast(ea, C.POINTER(C.c_double))
        rc = sfgmres_solve_batch(self.h, nrhs, b, x0, out, m, s, k, tol, SOLVE_TRANSPOSE if transpose else 0, st)
        info = {"status": rc, "problems": st.problems, "lockstep_outer": st.lockstep_outer,
                "total_inner": st.total_inner, "status_p": list(sa), "outer_iters_p": list(oa),
                "rel_res_true_p": list(ra), "rel_res_est_p": list(ea), "inner_steps_p": list(ka),
                "kernel_launches": st.kernel_launches,
                "t_total_ms": st.t_total_ms}
        return out, info

    def autotune(self, *, m: int, s: int, k: int, nrhs: int = 1):
        """Pick the row-block size and SpMV width by timing short inner cycles; returns ``(block_rows, spmv_vector,
        step_ms)``."""
        return sfgmres_autotune(self.h, nrhs, m, s, k)

    def update_values(self, vals) -> None:
        """Replace the stored values of A (same pattern and order)."""
        sfgmres_update_values(self.h, vals)

    def pattern_outer(self, u, v, alpha: float, out) -> None:
        """out[p] += alpha * u[row(p)] * v[col(p)] over the stored entries of A."""
        sfgmres_pattern_outer(self.h, u, v, alpha, out)

    def solve_restarted(self, b, x0=None, *, m: int, s: int, k: int, tol: float = 1e-8, max_cycles: int = 50,
                        out=None):
        """Restarted sGMRES (Algorithm 2) on ``b`` (CUDA tensor or NumPy array); returns ``(x, info)`` with the
        residual history ``||r_c|| / ||b||`` for c = 0 .. cycles."""
        import torch

        if out is None:
            out = torch.empty_like(b) if hasattr(b, "data_ptr") else np.empty_like(b)
        hist = np.zeros(max_cycles + 1, dtype=np.float64)
        rc, cycles = sfgmres_solve_restarted(self.h, b, x0, out, m, s, k, tol, max_cycles, hist)
        return out, {"status": rc, "cycles": cycles, "rel_res_hist": list(hist[:cycles + 1])}

    def inner_cycle(self, v, *, m: int, s: int, k: int, basis: bool = True):
        """One sGMRES cycle on the unit CUDA vector ``v``; returns ``(z, k, reason, basis[(m+1), n] or None, y)``."""
        import torch

        z = torch.empty_like(v)
        B = torch.zeros((m + 1, self.n), dtype=torch.float64, device=v.device) if basis else None
        y = torch.zeros(m, dtype=torch.float64, device=v.device)
        _, kk, rr = sfgmres_inner_cycle(self.h, v, z, m, s, k, B, y)
        return z, kk, rr, B, y[:kk]

    def precond_info(self):
        """``(colour int32[n], ncolours, lu float64[nnz])`` of the ILU(0) preconditioner (see sfgmres_precond_info)."""
        colour = np.empty(self.n, dtype=np.int32)
        lu = np.empty(self.nnz, dtype=np.float64)
        nc = sfgmres_precond_info(self.h, colour, lu)
        return colour, nc, lu

    def sketch(self, v, s: int):
        import torch

        c = torch.empty(s, dtype=torch.float64, device=v.device)
        sfgmres_sketch_apply(self.h, s, v, c)
        return c

    def sketch_pattern(self, s: int, device="cuda"):
        import torch

        zeta = 1 if self.get("sketch_kind") == 1 else int(self.get("zeta"))
        rows = torch.empty(self.n * zeta, dtype=torch.int32, device=device)
        signs = torch.empty(self.n * zeta, dtype=torch.int8, device=device)
        sfgmres_sketch_pattern(self.h, s, rows, signs)
        return rows.view(self.n, zeta), signs.view(self.n, zeta)

    def spmv(self, x):
        import torch

        y = torch.empty_like(x)
        sfgmres_spmv(self.h, x, y)
        return y

    def close(self) -> None:
        if getattr(self, "h", None):
            sfgmres_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
