"""Explicit low-precision rounding for the precision-matched inner cycle (oracle side).  TEST INFRASTRUCTURE ONLY.

The inner sGMRES cycle may run in FP32 (values, basis, sketch, dot products and their accumulation all FP32) or with
the basis *stored* in BF16 (arithmetic still FP32).  The outer FGMRES of Algorithm 1, the sketched QR and the
least-squares solve stay FP64.  NumPy has no BF16 type, so BF16 storage is emulated by rounding FP32 values to the
nearest BF16 value (ties to even) and keeping them in FP32 containers.
"""
from __future__ import annotations

import numpy as np

INNER_DTYPES = {"fp64": np.float64, "fp32": np.float32, "bf16": np.float32}


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16 value, ties to even (NaN stays NaN); returns FP32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    bits = x.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    rounded = ((bits + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    nan = np.isnan(x)
    out = rounded.view(np.float32).copy()
    out[nan] = np.float32(np.nan)
    return out


def store(x: np.ndarray, inner: str) -> np.ndarray:
    """Round a vector to the storage format of the inner basis."""
    if inner == "fp64":
        return np.asarray(x, dtype=np.float64)
    x32 = np.asarray(x, dtype=np.float32)
    if inner == "fp32":
        return x32
    if inner == "bf16":
        return round_bf16(x32)
    raise ValueError(inner)
