"""Pins of the quantisation oracle (Sec. 3.3 A) to facts that do not come from
the oracle itself: IEEE binary16 bit patterns from the standard, numpy's own
float16 conversion, closed forms of a uniform quantiser with an integer grid,
its error bound and monotonicity, and the straight-through QAT step against a
hand composition on a tiny case."""

import numpy as np
import pytest

from oracle import quant as Q


def test_half_bits_textbook_patterns():
    # IEEE 754 binary16: exponent bias 15, 10 fraction bits
    cases = [(1.0, 0x3C00), (-2.0, 0xC000), (0.5, 0x3800), (65504.0, 0x7BFF),
             (2.0 ** -14, 0x0400),
             (2.0 ** -24, 0x0001), (2.0 ** -25, 0x0000), (3 * 2.0 ** -25, 0x0002),
             (0.0, 0x0000), (-0.0, 0x8000), (65520.0, 0x7C00), (1e9, 0x7C00),
             (-np.inf, 0xFC00),
             (1.0 + 2.0 ** -11, 0x3C00),        # tie: to even (fraction 0)
             (1.0 + 3 * 2.0 ** -11, 0x3C02),    # tie: to even (fraction 2)
             (1.0 / 3.0, 0x3555), (2047.0, 0x67FF), (2049.0, 0x6800)]
    x = np.array([c[0] for c in cases], np.float32)
    np.testing.assert_array_equal(Q.half_bits(x), np.array([c[1] for c in cases], np.uint16))
    assert Q.half_bits(np.float32(np.nan)) == 0x7E00


def test_half_bits_match_numpy_float16():
    rng = np.random.default_rng(0)
    e = rng.uniform(-30, 17, 200000)
    x = (rng.choice([-1.0, 1.0], e.size) * rng.uniform(1, 2, e.size) * 2.0 ** e).astype(np.float32)
    # ties on the half grid at every exponent, and both ends of the ranges
    k = np.arange(-24, 16)
    ties = np.concatenate([(1 + (2 * j + 1) * 2.0 ** -11) * 2.0 ** k for j in range(4)])
    x = np.concatenate([x, ties.astype(np.float32), -ties.astype(np.float32),
                        np.float32([65503.9, 65519.99, 65520.0, 6.1e-5, 5.96e-8, 2.98e-8])])
    want = x.astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(Q.half_bits(x), want)
    np.testing.assert_array_equal(Q.half_value(want), x.astype(np.float16).astype(np.float32))


def test_half_value_roundtrip_every_pattern():
    b = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    v = Q.half_value(b)
    np.testing.assert_array_equal(np.isnan(v), np.isnan(b.view(np.float16)))
    fin = ~np.isnan(v)
    np.testing.assert_array_equal(v[fin], b.view(np.float16)[fin].astype(np.float32))
    np.testing.assert_array_equal(Q.half_bits(v[fin]), b[fin])


def test_uniform_integer_grid_closed_form():
    # lo = 0, hi = 255, 8 bits: scale = step = 1, code = rint(x) clamped
    bits = [8] + [0] * 8
    x = np.zeros((9, 9), np.float32)
    x[0] = [-3.0, 0.0, 0.49, 0.5, 1.5, 2.5, 254.6, 255.0, 300.0]
    codes, vals, ranges = Q.quantize(x, bits, [0.0] * 9, [255.0] * 9)
    np.testing.assert_array_equal(codes[0], [0, 0, 0, 0, 2, 2, 255, 255, 255])
    np.testing.assert_array_equal(vals[0], codes[0].astype(np.float32))
    np.testing.assert_array_equal(vals[1:], x[1:])        # float32 rows kept
    assert not codes[1:].any()
    assert tuple(ranges[:, 0]) == (0.0, 255.0)


@pytest.mark.parametrize("b", [1, 3, 6, 8, 10, 12, 16])
def test_uniform_error_bound_and_monotone(b):
    rng = np.random.default_rng(b)
    lo, hi = -1.7, 3.2
    x = np.sort(rng.uniform(lo, hi, 20000)).astype(np.float32)
    p = np.tile(x, (9, 1))
    bits = [b] * 9
    codes, vals, _ = Q.quantize(p, bits, [lo] * 9, [hi] * 9)
    c = codes[0].astype(np.int64)
    assert np.all(np.diff(c) >= 0)                       # monotone
    assert c.min() >= 0 and c.max() <= (1 << b) - 1
    step = (hi - lo) / ((1 << b) - 1)
    err = np.abs(vals[0].astype(np.float64) - x)
    # half a step plus float32 rounding of the affine map
    assert err.max() <= 0.5 * step + 8 * np.finfo(np.float32).eps * max(abs(lo), abs(hi))
    # the grid ends are exact codes: lo -> 0, hi -> 2^b - 1
    cl, vl, _ = Q.quantize(np.full((9, 2), [lo, hi], np.float32), bits, [lo] * 9, [hi] * 9)
    np.testing.assert_array_equal(cl[0], [0, (1 << b) - 1])
    assert vl[0, 0] == np.float32(lo)


def test_refine_ranges_are_the_row_extremes():
    rng = np.random.default_rng(5)
    p = rng.normal(0, 3, (9, 1000)).astype(np.float32)
    p[4, 17] = np.nan
    p[4, 18] = np.inf
    p[6] = 0.25                                          # no spread
    bits = [Q.HALF, Q.HALF, 6, 6, 6, 8, 8, 8, 0]
    codes, vals, ranges = Q.quantize(p, bits, refine=True)
    for r in (2, 3, 4, 5, 7):
        fin = p[r][np.isfinite(p[r])]
        assert (ranges[0, r], ranges[1, r]) == (fin.min(), fin.max())
        assert codes[r][np.argmin(np.where(np.isfinite(p[r]), p[r], np.inf))] == 0
        assert codes[r][np.argmax(np.where(np.isfinite(p[r]), p[r], -np.inf))] == (1 << bits[r]) - 1
    assert codes[4, 17] == 0 and codes[4, 18] == 0       # non-finite coded 0
    assert not codes[6].any() and np.all(vals[6] == np.float32(0.25))
    assert np.all(ranges[:, [0, 1, 8]] == 0)
    np.testing.assert_array_equal(vals[8], p[8])


def test_bits_per_gaussian():
    assert Q.bits_per_gaussian([Q.HALF, Q.HALF, 6, 6, 6, 8, 8, 8, 0]) == 32 + 18 + 24 + 32
    assert Q.bits_per_gaussian([0] * 9) == 9 * 32


def test_qat_step_is_straight_through_adam_at_quantised_values(oracle):
    from gs2d_inputs import random_gaussians, smooth_noise_target
    W, H, n = 24, 20, 6
    p = random_gaussians(n, W, H, seed=3, l_range=(1.5, 4.0))
    t = smooth_noise_target(W, H, seed=4)
    bits = [Q.HALF, Q.HALF, 4, 4, 4, 3, 3, 3, 4]
    m = np.zeros((9, n))
    v = np.zeros((9, n))
    p1, _, _, loss, grad = Q.qat_step(p, t, m, v, 1, bits, refine=True)
    _, pq, _ = Q.quantize(p, bits, refine=True)
    assert not np.array_equal(pq, p.astype(np.float32))
    # the gradient at the quantised parameters, by central differences of the
    # L2 loss of the brute-force render (a first Adam step moves each
    # parameter by lr against the sign of its gradient)
    h = 1e-4
    fd = np.zeros((9, n))
    base = pq.astype(np.float64)
    for r in range(9):
        for i in range(n):
            a, b = base.copy(), base.copy()
            a[r, i] += h
            b[r, i] -= h
            la = oracle.l2_loss(oracle.render(a, W, H), t)[0]
            lb = oracle.l2_loss(oracle.render(b, W, H), t)[0]
            fd[r, i] = (la - lb) / (2 * h)
    assert loss == pytest.approx(oracle.l2_loss(oracle.render(base, W, H), t)[0], rel=1e-12)
    np.testing.assert_allclose(grad, fd, rtol=1e-4, atol=1e-7)
    # and not the gradient at the float parameters
    at_p = np.zeros((9, n))
    p64 = p.astype(np.float64)
    for r in range(9):
        for i in range(n):
            a, b = p64.copy(), p64.copy()
            a[r, i] += h
            b[r, i] -= h
            at_p[r, i] = (oracle.l2_loss(oracle.render(a, W, H), t)[0]
                          - oracle.l2_loss(oracle.render(b, W, H), t)[0]) / (2 * h)
    assert np.abs(at_p - fd).max() > 100 * np.abs(grad - fd).max()
    # Adam's first step: lr g / (|g| + eps) on the float parameters
    moved = p1 - p64
    np.testing.assert_allclose(moved, -1e-2 * fd / (np.abs(fd) + 1e-8), rtol=1e-3, atol=1e-9)
