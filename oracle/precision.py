"""O7: numpy model of split-BF16 products (predicts, does not define, GPU error).

A float is split into bfloat16 pieces by round-to-nearest-even:
    x32 = fl32(x);  hi = bf16(x32);  mid = bf16(x32 - hi);  lo = bf16(x32 - hi - mid)
so hi + mid + lo == x32 exactly (each residual is exact in float32).
The product a b is approximated by the pieces' cross terms with
i + j <= 2 (six products) or i + j <= 1 (three products).  Bit-level
rounding below follows the IEEE-754 definition of round-to-nearest-even on
the float32 bit pattern.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32)
    # NaN/Inf pass through unchanged
    bad = ~np.isfinite(x)
    if np.any(bad):
        out = np.where(bad, x, out)
    return out


def split3(x):
    """(hi, mid, lo) float32 arrays holding bfloat16 values with hi + mid + lo == fl32(x)."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    hi = bf16_round(x32)
    r1 = (x32 - hi).astype(np.float32)
    mid = bf16_round(r1)
    r2 = (r1 - mid).astype(np.float32)
    lo = bf16_round(r2)
    return hi, mid, lo


def split_matmul(A, B, products: int = 6):
    """sum_{i+j<=p} A_i @ B_j with the products in float64 (the split error alone)."""
    Ap = split3(A)
    Bp = split3(B)
    pairs = [(0, 0), (0, 1), (1, 0)] if products == 3 else [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)]
    C = np.zeros((np.asarray(A).shape[0], np.asarray(B).shape[1]))
    for i, j in pairs:
        C += Ap[i].astype(np.float64) @ Bp[j].astype(np.float64)
    return C
