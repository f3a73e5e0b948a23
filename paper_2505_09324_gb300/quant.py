"""Quantisation of fitted Gaussians (Sec. 3.3 A) through libgs2d.

Per parameter row (mu_x, mu_y, l1, l2, l3, c_r, c_g, c_b, w) a quantiser is
IEEE half (``HALF``), float32 (0) or a uniform scalar quantiser of 1 ... 16
bits over a range.  The paper keeps distinct quantisers for the mean, the
Cholesky factor and the colour and adopts GaussianImage's without stating
them; ``DEFAULT_BITS`` is this library's choice, from a sweep on fitted
1080p conferencing frames: 16-bit uniform means (IEEE half spaces pixel
coordinates above 1024 a whole pixel apart, which cost 4-7 dB), 10-bit
Cholesky factor, 8-bit colour and weight: 94 bits per Gaussian, within
0.2-0.4 dB of the float fit.

* Post-training quantisation (PTQ): ``Quantizer.calibrate`` derives the
  ranges once, offline, from representative fitted frames (the training
  stage); ``Quantizer.quantize`` then codes a fitted frame in one kernel.
* Quantisation-aware fitting (QAT): ``GaussianRasterizer.encode_frame_qat``
  renders the quantised Gaussians inside every fit iteration
  (gs2d_fit_step_qat, straight-through gradient) with ranges re-derived from
  the current Gaussians at each step (``refine``).
* Bitstream accounting (Sec. 3.3 B, Eq. 3-4): ``code_bits`` (ideal order-0
  code length of the codes, per row, on the device), ``frame_bits`` (an I-
  or P-frame's coded size) and ``sequence_bits`` (bits-back totals).
"""

from __future__ import annotations

import numpy as np
import torch

from . import _native as nat

HALF = -16
ROWS = ("mu_x", "mu_y", "l1", "l2", "l3", "c_r", "c_g", "c_b", "w")
DEFAULT_BITS = (16, 16, 10, 10, 10, 8, 8, 8, 8)


class Quantizer:
    """Quantiser spec (bits per row; ranges for the uniform rows unless
    ``refine``) and the device call that applies it."""

    def __init__(self, bits=DEFAULT_BITS, lo=None, hi=None, refine: bool = False):
        bits = tuple(int(b) for b in bits)
        if len(bits) != 9 or any(not (b == HALF or 0 <= b <= 16) for b in bits):
            raise ValueError(f"bits must be 9 values in {{{HALF}, 0 ... 16}}: {bits}")
        uniform = [r for r in range(9) if bits[r] > 0]
        if uniform and not refine:
            if lo is None or hi is None:
                raise ValueError("uniform rows need lo and hi (or refine=True)")
            for r in uniform:
                if not (np.isfinite(lo[r]) and np.isfinite(hi[r]) and hi[r] > lo[r]):
                    raise ValueError(f"row {ROWS[r]}: range [{lo[r]}, {hi[r]}]")
        self.bits, self.refine = bits, bool(refine)
        self.lo = None if lo is None else tuple(float(np.float32(x)) for x in lo)
        self.hi = None if hi is None else tuple(float(np.float32(x)) for x in hi)
        self.c = nat.make_quant(bits, self.lo, self.hi, refine)

    @classmethod
    def calibrate(cls, param_sets, bits=DEFAULT_BITS, coverage: float = 1.0, stream=None):
        """PTQ calibration (Sec. 3.3 A): the range of every uniform row is the
        central ``coverage`` quantile interval of that row over the fitted
        frames in ``param_sets`` ([9, n] tensors or arrays), found on the
        device (gs2d_quant_calibrate); the default is the whole span (clipping
        the tails, at 99.9 %, cost 1.6 dB on fitted 1080p frames: the largest
        Gaussians matter).  A training-stage step that runs once per codec,
        not per frame; it synchronises the stream."""
        dev = next((p.device for p in param_sets
                    if isinstance(p, torch.Tensor) and p.is_cuda), torch.device("cuda"))
        rows = [(p.detach() if isinstance(p, torch.Tensor) else torch.from_numpy(
            np.ascontiguousarray(p, np.float32))).to(dev, torch.float32).reshape(9, -1)
            for p in param_sets]
        allp = torch.cat(rows, dim=1).contiguous()
        nbytes = int(nat.load().gs2d_quant_calibrate_scratch_bytes())
        scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        s = torch.cuda.current_stream(dev) if stream is None else stream
        lo, hi = nat.quant_calibrate(allp.data_ptr(), allp.shape[1], bits, coverage,
                                     scratch.data_ptr(), nbytes, int(s.cuda_stream))
        return cls(bits, lo, hi)

    @property
    def bits_per_gaussian(self) -> int:
        """Payload bits per Gaussian (16 per half row, b per uniform row, 32
        per float32 row)."""
        return int(sum(16 if b == HALF else (32 if b == 0 else b) for b in self.bits))

    def frame_bytes(self, n: int) -> int:
        """Bytes of one coded frame of n Gaussians: the packed codes plus the
        ranges (two float32 per uniform row)."""
        return (n * self.bits_per_gaussian + 7) // 8 + 8 * sum(b > 0 for b in self.bits)

    def quantize(self, params: torch.Tensor, codes: bool = True, values: bool = True,
                 stream=None):
        """gs2d_quantize: (codes uint16 [9, n] | None, dequantised float32
        [9, n] | None, ranges float32 [2, 9])."""
        if not (isinstance(params, torch.Tensor) and params.is_cuda
                and params.dtype == torch.float32 and params.is_contiguous()
                and params.dim() == 2 and params.shape[0] == 9):
            raise ValueError("params must be a contiguous float32 CUDA tensor [9, n]")
        if not (codes or values):
            raise ValueError("ask for codes, values or both")
        n = params.shape[1]
        c = torch.empty((9, n), dtype=torch.uint16, device=params.device) if codes else None
        v = torch.empty_like(params) if values else None
        ranges = torch.empty((2, 9), dtype=torch.float32, device=params.device)
        s = torch.cuda.current_stream() if stream is None else stream
        nat.quantize(params.data_ptr(), n, self.c, 0 if c is None else c.data_ptr(),
                     0 if v is None else v.data_ptr(), ranges.data_ptr(), int(s.cuda_stream))
        return c, v, ranges


_scratch = {}


def code_bits(codes: torch.Tensor, bits, select: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
    """gs2d_code_entropy: ideal order-0 code length (bits, float64 [9] on the
    device) of each row of the [9, n] codes, over the selected columns."""
    n = codes.shape[1]
    dev = codes.device
    nbytes = int(nat.load().gs2d_code_entropy_scratch_bytes())
    buf = _scratch.get(dev)
    if buf is None or buf.numel() < nbytes:
        buf = _scratch[dev] = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = torch.empty(9, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream(dev) if stream is None else stream
    nat.code_entropy(codes.data_ptr(), n, bits, 0 if select is None else select.data_ptr(),
                     buf.data_ptr(), nbytes, out.data_ptr(), int(s.cuda_stream))
    return out


def frame_bits(quantizer: Quantizer, params: torch.Tensor, select: torch.Tensor | None = None,
               stream=None) -> float:
    """Coded size of a frame (gs2d_frame_bits; host float, synchronises):
    the entropy-coded codes of all Gaussians (an I-frame) or of the selected
    ones, each with its index of ceil(log2 n) bits (a P-frame), plus the
    frame's ranges (two float32 per uniform row) when the quantiser refines
    them per frame."""
    codes, _, _ = quantizer.quantize(params, values=False, stream=stream)
    n = params.shape[1]
    dev = params.device
    nbytes = int(nat.load().gs2d_frame_bits_scratch_bytes())
    key = (dev, "frame")
    buf = _scratch.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = _scratch[key] = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream(dev) if stream is None else stream
    b = (nat.ctypes.c_int32 * 9)(*quantizer.bits)
    nat.check(nat.load().gs2d_frame_bits(
        nat._p(codes.data_ptr()), n, b, nat._p(0 if select is None else select.data_ptr()),
        int(quantizer.refine), nat._p(buf.data_ptr()), nbytes, nat._p(out.data_ptr()),
        nat._p(int(s.cuda_stream))), "gs2d_frame_bits")
    return float(out.item())


def sequence_bits(counts, payload_bits, gop: int) -> dict:
    """gs2d_sequence_bits: I-frame bits, P-frame bits, bits-back savings
    (Eq. 3 per P-frame, Eq. 4 summed) and the total of a coded sequence."""
    return nat.sequence_bits(counts, payload_bits, gop)
