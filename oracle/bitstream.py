"""Oracle for the bitstream accounting of a coded sequence (Sec. 3.3 B,
Eq. 3-4) -- TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper sends every I-frame (the first frame of each group of pictures)
with vanilla entropy coding of all N Gaussians, and every P-frame as the
subset of Gaussians that were re-fitted, with bits-back coding, whose saving
per P-frame is log((m)!) - log(m) for m coded Gaussians (Eq. 3; the paper
writes m = N/20, its average) and (F - F/K) S_P over a sequence of F frames
with an I-frame every K frames (Eq. 4).  Readings (the paper fixes none of
them): logarithms are base 2 (bits); the I-frame interval K counts frames
(frame k is an I-frame when k mod K = 0); a P-frame Gaussian carries its
index, ceil(log2 N) bits, next to its codes (the decoder must know which
Gaussians changed; bits-back reclaims the order of that set); the vanilla
entropy coder is an ideal order-0 coder with one static model per parameter
row, whose length is the empirical entropy of the row's codes (a bound any
real coder of that model approaches, model cost not counted).
"""

from __future__ import annotations

import math

import numpy as np


def log2_factorial(m: int) -> float:
    """log2(m!) as the plain sum of log2(k) for k = 2 ... m."""
    return float(sum(math.log2(k) for k in range(2, int(m) + 1)))


def bitsback_saving(m: int) -> float:
    """Eq. 3: bits saved by bits-back coding of a P-frame that codes m
    Gaussians, log2(m!) - log2(m); 0 for m <= 1."""
    m = int(m)
    if m <= 1:
        return 0.0
    return log2_factorial(m) - math.log2(m)


def code_entropy_bits(codes, bits, select=None) -> np.ndarray:
    """Ideal order-0 code length, per parameter row, of [9, n] codes (only the
    columns with select[i] != 0 when select is given): the sum over the
    row's distinct symbols s of -c_s log2(c_s / n).  Rows kept as float32
    (bits 0) count 32 bits per value; IEEE-half rows are coded like the
    others (16-bit symbols)."""
    c = np.asarray(codes, np.uint16).reshape(9, -1)
    if select is not None:
        c = c[:, np.asarray(select).astype(bool)]
    n = c.shape[1]
    out = np.zeros(9)
    for r in range(9):
        if int(bits[r]) == 0:
            out[r] = 32.0 * n
            continue
        if n == 0:
            continue
        _, counts = np.unique(c[r], return_counts=True)
        out[r] = float(sum(-k * math.log2(k / n) for k in counts))
    return out


def sequence_bits(counts, payload_bits, K: int):
    """Eq. 3-4 over a sequence of F frames.  counts[k] = Gaussians coded in
    frame k; payload_bits[k] = its coded size before bits-back (an I-frame:
    the vanilla entropy-coded Gaussians; a P-frame: its coded Gaussians with
    their indices).  Frame k is an I-frame when k mod K = 0; every P-frame
    saves bitsback_saving(counts[k]).  Returns the I-frame bits, the P-frame
    bits before bits-back, the total saving and the total."""
    F = len(counts)
    i_bits = p_bits = saving = 0.0
    for k in range(F):
        if k % K == 0:
            i_bits += float(payload_bits[k])
        else:
            p_bits += float(payload_bits[k])
            saving += bitsback_saving(counts[k])
    return {"i_bits": i_bits, "p_bits": p_bits, "savings": saving,
            "total_bits": i_bits + p_bits - saving,
            "i_frames": sum(1 for k in range(F) if k % K == 0),
            "p_frames": sum(1 for k in range(F) if k % K != 0)}
