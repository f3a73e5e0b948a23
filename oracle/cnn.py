"""Oracle for the learned initialiser (Sec. 3.2 B: a regressor from the frame
to the Gaussians' parameters, trained with a Chamfer loss) -- TEST
INFRASTRUCTURE ONLY (see the package docstring).

Plain double-precision numpy: BF16 rounding written from its bit-level
definition, matrix products, convolutions as explicit sums over the 3 x 3
taps, the head's decoding of a network output into Gaussians, and the
Chamfer distance by brute force.
"""

from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Rounds float32 values to the nearest bfloat16 (ties to even), returned as
    float32: keep the upper 16 bits of the IEEE single after adding
    0x7FFF + (bit 16) to the lower half.  NaN stays NaN."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out)


def bf16_bits(x) -> np.ndarray:
    """uint16 bit patterns of bf16_round(x)."""
    return (bf16_round(x).view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def gemm(a, b, bias=None, relu=False) -> np.ndarray:
    """C = A B^T (+ bias, then max(., 0)) in double precision; A [M, K], B [N, K]."""
    c = np.asarray(a, np.float64) @ np.asarray(b, np.float64).T
    if bias is not None:
        c = c + np.asarray(bias, np.float64)[None, :]
    if relu:
        c = np.maximum(c, 0.0)
    return c


def gemm_abs(a, b) -> np.ndarray:
    """sum_k |A[m, k] B[n, k]|: the scale of the rounding error of C[m, n]."""
    return np.abs(np.asarray(a, np.float64)) @ np.abs(np.asarray(b, np.float64)).T
