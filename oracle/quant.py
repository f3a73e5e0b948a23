"""Oracle for the quantisation of fitted Gaussians (Sec. 3.3 A) -- TEST
INFRASTRUCTURE ONLY (see the package docstring).

The paper keeps distinct quantisers for the mean, the Cholesky factor and the
colour and takes them from GaussianImage without stating them; the readings
used here: a row either stays float32, is stored as IEEE half, or goes through
a uniform scalar quantiser of b bits over a range [lo, hi].  Post-training
quantisation (PTQ) takes the range from calibration over representative
fitted frames; quantisation-aware fitting (QAT) renders the quantised
Gaussians inside the fit loop, passes the gradient straight through to the
float parameters, and re-derives every range from the current parameters at
each step ("refine": [min, max] of the row).

Integer codes are decided by floating point, so the uniform quantiser is
evaluated in the precision the kernel uses: single-rounded float32
operations (numpy float32 arithmetic), with scale and step formed in double
and rounded once to float.  The half conversion is written from its
definition (round to nearest, ties to even, on the 11-bit significand grid).
"""

from __future__ import annotations

import numpy as np

HALF = -16
ROWS = 9


def half_bits(x) -> np.ndarray:
    """IEEE binary16 bit patterns of float32 values, rounded to nearest with
    ties to even.  A finite |x| < 2^-14 is a subnormal with code
    rint(|x| 2^24); otherwise, with e = floor(log2 |x|) <= 15, the code is
    ((e + 15) << 10) + rint(|x| 2^(10 - e)) - 1024 (a significand that rounds
    up to 2048 carries into the exponent, and past e = 15 gives infinity);
    larger values and infinities give 0x7C00; NaN gives 0x7E00 with the sign
    dropped."""
    a = np.atleast_1d(np.asarray(x, np.float32)).astype(np.float64)
    shape = np.shape(x)
    sign = np.signbit(a).astype(np.uint32) << 15
    mag = np.abs(a)
    out = np.zeros(a.shape, np.uint32)
    with np.errstate(divide="ignore", invalid="ignore"):
        fin = np.isfinite(mag)
        sub = fin & (mag < 2.0 ** -14)
        out[sub] = np.rint(mag[sub] * 2.0 ** 24).astype(np.uint32)
        nrm = fin & ~sub
        e = np.floor(np.log2(np.where(nrm, mag, 1.0)))
        # log2 of a float32 can land a hair off an integer: fix e so that
        # 2^e <= |x| < 2^(e+1) holds exactly
        e = np.where(np.ldexp(1.0, e.astype(np.int64)) > mag, e - 1, e)
        e = np.where(np.ldexp(1.0, (e + 1).astype(np.int64)) <= mag, e + 1, e)
        big = nrm & (e > 15)
        ok = nrm & ~big
        sig = np.rint(np.ldexp(mag, (10 - e).astype(np.int64)))
        code = (e + 15) * 1024 + sig - 1024
        out[ok] = code[ok].astype(np.uint32)
        out[big] = 0x7C00
        out[np.isinf(mag)] = 0x7C00
    out = out | sign
    out[np.isnan(a)] = 0x7E00
    return out.astype(np.uint16).reshape(shape)


def half_value(bits) -> np.ndarray:
    """float32 value of binary16 bit patterns: (-1)^s m 2^-24 for exponent
    field 0, (-1)^s (1024 + m) 2^(E - 25) for E in 1 ... 30, infinity or NaN
    for E = 31."""
    b = np.asarray(bits, np.uint16).astype(np.int64)
    s = np.where(b >> 15, -1.0, 1.0)
    E = (b >> 10) & 31
    m = b & 1023
    v = np.where(E == 0, m * 2.0 ** -24, np.ldexp((1024 + m).astype(np.float64), E - 25))
    v = np.where(E == 31, np.where(m == 0, np.inf, np.nan), v)
    return (s * v).astype(np.float32)


def scale_step(bits: int, lo, hi):
    """scale = (2^b - 1) / (hi - lo) and step = (hi - lo) / (2^b - 1),
    evaluated in double from the float32 range and rounded to float32; both 0
    when hi <= lo."""
    lo64, hi64 = float(np.float32(lo)), float(np.float32(hi))
    if not hi64 > lo64:
        return np.float32(0.0), np.float32(0.0)
    levels = float((1 << bits) - 1)
    d = hi64 - lo64
    return np.float32(levels / d), np.float32(d / levels)


def quantize(params, bits, lo=None, hi=None, refine: bool = False):
    """Quantises the [9, n] parameters row by row (Sec. 3.3 A).

    bits[r] = -16: IEEE half (``half_bits``); 0: float32 kept, code 0;
    1 ... 16: code = clamp(rint((x - lo) scale), 0, 2^b - 1) and value
    lo + code step in float32, non-finite x coded 0.  With ``refine`` the range
    of each uniform row is [min, max] of its finite values (lo = hi = 0 when it
    has none).  Returns (codes uint16 [9, n], values float32 [9, n],
    ranges float32 [2, 9] with the lo and hi of the uniform rows)."""
    x = np.asarray(params, np.float32).reshape(ROWS, -1)
    n = x.shape[1]
    codes = np.zeros((ROWS, n), np.uint16)
    values = x.copy()
    ranges = np.zeros((2, ROWS), np.float32)
    for r in range(ROWS):
        b = int(bits[r])
        row = x[r]
        if b == HALF:
            codes[r] = half_bits(row)
            values[r] = half_value(codes[r])
        elif b > 0:
            if refine:
                fin = row[np.isfinite(row)]
                lo_r = fin.min() if fin.size else np.float32(0.0)
                hi_r = fin.max() if fin.size else np.float32(0.0)
            else:
                lo_r, hi_r = lo[r], hi[r]
            lo_r, hi_r = np.float32(lo_r), np.float32(hi_r)
            scale, step = scale_step(b, lo_r, hi_r)
            with np.errstate(invalid="ignore", over="ignore"):
                k = np.rint((row - lo_r) * scale)
            k = np.where(np.isfinite(row), k, np.float32(0.0))
            k = np.clip(k, np.float32(0.0), np.float32((1 << b) - 1)).astype(np.float32)
            codes[r] = k.astype(np.uint16)
            values[r] = lo_r + k * step
            ranges[:, r] = (lo_r, hi_r)
        elif b != 0:
            raise ValueError(f"bits[{r}] = {b}")
    return codes, values, ranges


def bits_per_gaussian(bits) -> int:
    """Payload bits of one Gaussian: 16 per half row, b per uniform row, 32
    per float32 row (the per-frame ranges, 2 floats per uniform row, come on
    top once per frame)."""
    return int(sum(16 if b == HALF else (32 if b == 0 else b) for b in bits))


def qat_step(params, target, m, v, step: int, bits, lo=None, hi=None, refine: bool = False,
             lr: float = 1e-2, cfg=None):
    """One quantisation-aware fit iteration (Sec. 3.3 A): quantise the float
    parameters, take the L2 loss gradient of Eq. 2 at the quantised values,
    pass it straight through (the quantiser's derivative is read as 1) and
    apply Adam to the float parameters.  Returns (params, m, v, loss, grad)."""
    from . import Config, adam_step, loss_and_grad
    _, pq, _ = quantize(np.asarray(params, np.float32), bits, lo, hi, refine)
    res = loss_and_grad(pq, target, cfg or Config())
    p, m, v = adam_step(np.asarray(params, np.float64), res["grad"], m, v, step, lr=lr)
    return p, m, v, res["loss"], res["grad"]
