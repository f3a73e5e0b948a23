"""Pins of the oracle's small helpers by brute force: the convolution output
size by enumerating window positions, the superpixel segment means and the
K-means update (paper Sec. 3.2 A) by explicit per-pixel loops, and the
quantiser's scale and step (Sec. 3.3 A) by the codes they give the range's
end points.  Each helper is also exercised through its caller's pins."""

import numpy as np
import pytest

from oracle import cnn, quant, superpixel as sp


@pytest.mark.parametrize("n", [1, 2, 5, 8, 17])
@pytest.mark.parametrize("ks,stride,pad", [(1, 1, 0), (3, 1, 1), (3, 2, 1), (5, 2, 2), (3, 3, 0),
                                           (2, 2, 0), (5, 2, 4)])
def test_out_size_counts_window_positions(n, ks, stride, pad):
    # output positions o whose window [o s - pad, o s - pad + ks) lies inside the
    # zero-padded input [-pad, n + pad)
    count = 0
    o = 0
    while o * stride - pad + ks <= n + pad:
        count += 1
        o += 1
    if n + 2 * pad < ks:                     # no window fits (the layers never ask)
        assert count == 0
        return
    assert cnn.out_size(n, ks, stride, pad) == count


def test_segment_means_by_loops():
    g = np.random.Generator(np.random.PCG64(3))
    h, w, k = 7, 9, 5
    frame = g.uniform(0, 1, size=(3, h, w)).astype(np.float32)
    label = g.integers(-1, k - 1, size=(h, w))   # label k - 1 stays empty; -1 = outside
    cnt, mxy, mc = sp.segment_means(frame, label, k)
    for s in range(k):
        px = [(x, y) for y in range(h) for x in range(w) if label[y, x] == s]
        assert cnt[s] == len(px)
        if not px:
            assert np.all(np.isnan(mxy[s])) and np.all(np.isnan(mc[s]))
            continue
        assert mxy[s, 0] == pytest.approx(sum(x + 0.5 for x, _ in px) / len(px), rel=1e-15)
        assert mxy[s, 1] == pytest.approx(sum(y + 0.5 for _, y in px) / len(px), rel=1e-15)
        for ch in range(3):
            ref = sum(float(frame[ch, y, x]) for x, y in px) / len(px)
            assert mc[s, ch] == pytest.approx(ref, rel=1e-14)


def test_update_moves_to_means_clamped_to_seed_window():
    g = np.random.Generator(np.random.PCG64(4))
    h, w, k, S = 12, 16, 4, 2.0
    frame = g.uniform(0, 1, size=(3, h, w)).astype(np.float32)
    label = np.full((h, w), -1)
    label[0:6, 0:8] = 0
    label[0:6, 8:16] = 1
    label[6:12, 0:16] = 2                      # segment 3 has no pixel
    seeds = np.array([[1.0, 1.0], [12.0, 3.0], [8.0, 9.0], [5.0, 5.0]])
    col0 = g.uniform(0, 1, size=(k, 3))
    xy0 = seeds + 0.25
    col, xy = sp.update(frame, label, col0, xy0, seeds, S)
    for s in range(3):
        ys, xs = np.nonzero(label == s)
        mx, my = (xs + 0.5).mean(), (ys + 0.5).mean()
        assert xy[s, 0] == pytest.approx(min(max(mx, seeds[s, 0] - S), seeds[s, 0] + S))
        assert xy[s, 1] == pytest.approx(min(max(my, seeds[s, 1] - S), seeds[s, 1] + S))
        np.testing.assert_allclose(col[s], frame[:, ys, xs].astype(np.float64).mean(1), rtol=1e-14)
    # segment 0's mean (4.0, 3.0) lies outside [seed -/+ S] on x: clamped to 3.0
    assert xy[0, 0] == 3.0
    # the empty segment keeps its centre
    np.testing.assert_array_equal(xy[3], xy0[3])
    np.testing.assert_array_equal(col[3], col0[3])


@pytest.mark.parametrize("bits", [1, 3, 6, 8, 12, 16])
@pytest.mark.parametrize("lo,hi", [(-1.5, 2.25), (0.0, 1.0), (-3e-3, 7e-2), (100.0, 100.5)])
def test_scale_step_codes_the_range_end_points(bits, lo, hi):
    scale, step = quant.scale_step(bits, lo, hi)
    levels = (1 << bits) - 1
    lo32, hi32 = np.float32(lo), np.float32(hi)
    # the range's ends take the first and the last code; values on the grid
    assert int(np.rint((np.float64(lo32) - np.float64(lo32)) * np.float64(scale))) == 0
    assert int(np.rint((np.float64(hi32) - np.float64(lo32)) * np.float64(scale))) == levels
    assert abs(float(lo32) + levels * float(step) - float(hi32)) <= 1e-6 * max(1.0, abs(hi))
    assert float(scale) * float(step) == pytest.approx(1.0, rel=1e-6)


def test_scale_step_of_an_empty_range():
    assert quant.scale_step(8, 1.0, 1.0) == (0.0, 0.0)
    assert quant.scale_step(8, 2.0, 1.0) == (0.0, 0.0)


def test_head_keys_read_each_slots_weight_channel():
    # out [B, gh gw, 9 slots]: slot s of cell c has its 9 outputs at 9 s ... 9 s + 8,
    # the weight offset last; key = |0.25 + o8| in float32
    B, gh, gw, slots = 2, 3, 4, 5
    g = np.random.Generator(np.random.PCG64(6))
    out = g.normal(size=(B, gh * gw, 9 * slots)).astype(np.float32)
    keys = cnn.head_keys(out, gh, gw, slots)
    assert keys.shape == (B, gh * gw * slots) and keys.dtype == np.float32
    for b in range(B):
        for c in range(gh * gw):
            for s in range(slots):
                ref = abs(np.float32(0.25) + out[b, c, 9 * s + 8])
                assert keys[b, c * slots + s] == ref


def test_initial_centres_take_the_seed_pixel():
    g = np.random.Generator(np.random.PCG64(7))
    frame = g.uniform(0, 1, size=(3, 6, 10)).astype(np.float32)
    sxy = np.array([[0.5, 0.5], [9.99, 5.99], [3.2, 4.0], [10.0, 6.0], [-0.3, 2.5]])
    col, xy = sp.initial_centres(frame, sxy)
    np.testing.assert_array_equal(xy, sxy)
    for i, (x, y) in enumerate(sxy):
        xi = min(max(int(np.floor(x)), 0), 9)   # positions on the edge clamp to the last pixel
        yi = min(max(int(np.floor(y)), 0), 5)
        np.testing.assert_array_equal(col[i], frame[:, yi, xi].astype(np.float64))
