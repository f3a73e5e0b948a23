"""Quantisation (Sec. 3.3 A) on the GPU against the oracle: PTQ codes, values
and ranges bit-exact (caller ranges and refined ranges, ragged and empty
sizes, non-finite inputs, the full 1080p Gaussian set), the QAT fit iteration
against the straight-through oracle iteration, and QAT against PTQ on the
quantised quality."""

import numpy as np
import pytest

from gs2d_inputs import (conferencing_frame, conferencing_gaussians, random_gaussians,
                         smooth_noise_target)
from oracle import quant as Q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED = [Q.HALF, Q.HALF, 6, 8, 10, 5, 8, 12, 16]


@pytest.fixture(scope="module")
def gs():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    import paper_2505_09324_gb300 as pkg
    return pkg


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def codes_np(t):
    return t.cpu().view(torch.int16).numpy().view(np.uint16)


def messy_params(n, seed):
    """Gaussians spread beyond the calibrated ranges, with NaN and infinities,
    values on the half grid's rounding ties and at the range ends."""
    rng = np.random.default_rng(seed)
    p = random_gaussians(n, 640, 360, seed=seed).astype(np.float32)
    p[2:] += rng.normal(0, 0.5, (7, n)).astype(np.float32)
    if n >= 8:
        p[3, 0], p[4, 1], p[5, 2] = np.nan, np.inf, -np.inf
        p[0, 3] = np.float32(1.0 + 2.0 ** -11)              # half tie
        p[1, 4] = np.float32(70000.0)                        # half overflow
        p[2, 5], p[2, 6] = -50.0, 50.0                       # clamped
    return p


def compare(gs, p, bits, lo=None, hi=None, refine=False):
    q = gs.Quantizer(bits, lo, hi, refine=refine)
    codes, vals, ranges = q.quantize(to_dev(p))
    torch.cuda.synchronize()
    oc, ov, orng = Q.quantize(p, bits, lo, hi, refine)
    np.testing.assert_array_equal(codes_np(codes), oc)
    np.testing.assert_array_equal(vals.cpu().numpy(), ov)       # NaN == NaN here
    np.testing.assert_array_equal(ranges.cpu().numpy(), orng)
    return oc


@pytest.mark.parametrize("n", [1, 7, 37, 1000, 20011])
def test_ptq_bit_exact_caller_ranges(gs, n):
    p = messy_params(n, seed=n)
    lo = [0, 0, 0.5, -2.0, 0.5, -0.2, -0.2, -0.2, 0.0]
    hi = [1, 1, 9.0, 2.0, 9.0, 1.2, 1.2, 1.2, 1.5]
    compare(gs, p, MIXED, lo, hi)


@pytest.mark.parametrize("n", [1, 7, 1000, 20011])
def test_ptq_bit_exact_refined_ranges(gs, n):
    p = messy_params(n, seed=100 + n)
    if n >= 8:
        p[6] = 0.25                  # a uniform row with no spread
        p[7] = np.nan                # a uniform row with no finite value
    compare(gs, p, MIXED, refine=True)


def test_ptq_every_width(gs):
    p = messy_params(5000, seed=9)
    for b in range(1, 17):
        compare(gs, p, [b] * 9, refine=True)
    compare(gs, p, [0] * 9)
    compare(gs, p, [Q.HALF] * 9)


def test_ptq_empty(gs):
    q = gs.Quantizer(MIXED, refine=True)
    codes, vals, ranges = q.quantize(torch.empty((9, 0), device="cuda"))
    torch.cuda.synchronize()
    assert codes.numel() == 0 and vals.numel() == 0


def test_ptq_full_size_1080p(gs):
    frame, mask = conferencing_frame(1920, 1080, seed=1)
    p = conferencing_gaussians(frame, mask, 20000, seed=2)
    q = gs.Quantizer.calibrate([p], MIXED)
    oc = compare(gs, p, MIXED, q.lo, q.hi)
    assert len(np.unique(oc[5])) > 20
    compare(gs, p, MIXED, refine=True)


def test_qat_with_identity_quantiser_is_the_fit_step(gs):
    from paper_2505_09324_gb300 import _native as nat
    W, H, n = 200, 120, 500
    p0 = to_dev(random_gaussians(n, W, H, seed=11, l_range=(2.0, 6.0)))
    t = to_dev(smooth_noise_target(W, H, seed=12))
    r = gs.GaussianRasterizer(W, H, n)
    s = int(torch.cuda.current_stream().cuda_stream)
    q = gs.Quantizer([0] * 9)
    a, b = p0.clone(), p0.clone()
    ma, va, mb, vb = (torch.empty_like(p0) for _ in range(4))
    nat.fit_reset(r.plan, r.ws_ptr, ma.data_ptr(), va.data_ptr(), s)
    nat.fit_reset(r.plan, r.ws_ptr, mb.data_ptr(), vb.data_ptr(), s)
    for _ in range(3):
        nat.fit_step(r.plan, r.ws_ptr, t.data_ptr(), a.data_ptr(), ma.data_ptr(), va.data_ptr(), s)
    nat.fit_reset(r.plan, r.ws_ptr, mb.data_ptr(), vb.data_ptr(), s)
    for _ in range(3):
        nat.fit_step_qat(r.plan, r.ws_ptr, t.data_ptr(), b.data_ptr(), mb.data_ptr(),
                         vb.data_ptr(), q.c, s)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(ma, mb) and torch.equal(va, vb)


@pytest.mark.parametrize("refine", [False, True])
def test_qat_loop_tracks_oracle(gs, oracle, refine):
    """64x64 frame, 50 Gaussians, 30 QAT iterations against the oracle's
    straight-through loop (quantise, gradient at the quantised values, Adam
    on the float parameters)."""
    W, H, n, iters = 64, 64, 50, 30
    bits = [Q.HALF, Q.HALF, 5, 5, 5, 4, 4, 4, 5]
    p0 = random_gaussians(n, W, H, seed=31, l_range=(2.0, 6.0))
    target = smooth_noise_target(W, H, seed=32)
    lo = [0, 0, 0.0, -4.0, 0.0, -0.5, -0.5, -0.5, 0.0]
    hi = [1, 1, 8.0, 4.0, 8.0, 1.5, 1.5, 1.5, 1.5]
    q = gs.Quantizer(bits, None if refine else lo, None if refine else hi, refine=refine)
    r = gs.GaussianRasterizer(W, H, n)
    tp = to_dev(p0)
    out = r.encode_frame_qat(to_dev(target), tp, iters, q)
    p = p0.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for it in range(1, iters + 1):
        p, m, v, _, _ = Q.qat_step(p, target, m, v, it, bits, lo, hi, refine)
    got = tp.cpu().numpy().astype(np.float64)
    _, pq_ref, _ = Q.quantize(p.astype(np.float32), bits, lo, hi, refine)
    l_ref = oracle.l2_loss(oracle.render(pq_ref, W, H), target)[0]
    _, pq_got, _ = Q.quantize(got.astype(np.float32), bits, lo, hi, refine)
    l_got = oracle.l2_loss(oracle.render(pq_got, W, H), target)[0]
    l_0 = oracle.l2_loss(oracle.render(p0, W, H), target)[0]
    assert abs(l_got - l_ref) <= 3e-2 * l_ref, (l_got, l_ref)
    assert l_ref < 0.5 * l_0
    scale = np.abs(p).max(axis=1, keepdims=True) + 1e-3
    assert np.median(np.abs(got - p) / scale) < 1e-3
    # the library's final quantisation is the oracle's of the same floats
    np.testing.assert_array_equal(codes_np(out["codes"]),
                                  Q.quantize(tp.cpu().numpy(), bits, lo, hi, refine)[0])


def test_qat_raises_the_quantised_quality_of_a_fit(gs):
    """QAT optimises the loss of the quantised Gaussians: 300 QAT iterations
    from a 300-iteration fit raise its 5-bit quantised PSNR (by 2.7-4.4 dB
    over five seeds).  At equal iteration counts plain fitting followed by
    PTQ does as well or better on these frames."""
    W, H, n = 256, 256, 800
    bits = [Q.HALF, Q.HALF, 5, 5, 5, 5, 5, 5, 5]
    target = to_dev(smooth_noise_target(W, H, seed=41, terms=24, max_cycles=8))
    p0 = to_dev(random_gaussians(n, W, H, seed=42, l_range=(3.0, 8.0)))
    r = gs.GaussianRasterizer(W, H, n)
    q = gs.Quantizer(bits, refine=True)
    ptq = p0.clone()
    r.encode_frame(target, ptq, 300, check_every=300)
    _, vals, _ = q.quantize(ptq)
    psnr_float, psnr_ptq = r.psnr(target, ptq), r.psnr(target, vals)
    qat = ptq.clone()
    out = r.encode_frame_qat(target, qat, 300, q)
    assert psnr_ptq < psnr_float - 0.5          # 5-bit codes cost quality
    assert out["psnr_q"] > psnr_ptq + 1.0, (psnr_float, psnr_ptq, out["psnr_q"])


@pytest.mark.parametrize("coverage", [1.0, 0.999, 0.5])
def test_ptq_calibration_is_the_quantile_interval(gs, coverage):
    """gs2d_quant_calibrate (order statistics by a device radix select,
    interpolated in double) against numpy's quantile of the finite values of
    every uniform row over several frames, non-finite values, duplicates and
    negative zeros included; a constant row gets hi = lo + 1."""
    rng = np.random.default_rng(3)
    sets = []
    for k, n in enumerate((5000, 1, 777)):
        p = rng.normal(0.0, 10.0 ** (k - 1), (9, n)).astype(np.float32)
        sets.append(p)
    sets[0][2, :50] = np.nan
    sets[0][3, :7] = np.inf
    sets[0][4, :9] = -np.inf
    sets[2][5, :100] = 0.25          # duplicates
    sets[2][6, :10] = -0.0
    for s in sets:
        s[7] = 3.5                    # a constant row
    bits = (8, 8, 8, 8, 8, 8, 8, 8, Q.HALF)
    q = gs.Quantizer.calibrate([torch.from_numpy(s).cuda() for s in sets], bits, coverage)
    allp = np.concatenate(sets, axis=1).astype(np.float64)
    lo_q = (1.0 - coverage) / 2.0
    for r in range(9):
        if bits[r] <= 0:
            continue
        x = allp[r][np.isfinite(allp[r])]
        lo, hi = np.quantile(x, lo_q), np.quantile(x, 1.0 - lo_q)
        if not hi > lo:
            hi = lo + 1.0
        assert q.lo[r] == float(np.float32(lo)) and q.hi[r] == float(np.float32(hi)), r
