"""Pins for the oracle's region-of-interest superpixel initialiser (Sec. 3.2 A:
superpixel centre -> mean, segment covariance -> Cholesky factor (Eq. 1), mean
colour -> colour), each against a closed form that a dropped term, a swapped
axis, a wrong sign or a quantised sum would break."""

import math

import numpy as np
import pytest

from gs2d_inputs import block_image, conferencing_frame, rng


def test_block_image_segments_are_the_blocks():
    """Constant-colour b x b blocks, seed step S = b: each block is a segment;
    its Gaussian has mean = block centre, Sigma = 4 (b^2/12) I (kappa = 4 times
    the second moment of a b x b square), colour = block colour exactly (the
    float32 value: the mean of equal values, no quantisation) and weight
    b^2 / (2 pi b^2/3) = 3/(2 pi)."""
    from oracle import superpixel as sp
    bx, by, b = 8, 6, 6
    img, cols = block_image(bx, by, b)
    mask = np.ones(img.shape[1:], bool)
    n = bx * by
    params, info = sp.roi_init(img, mask, n, 1.0, np.zeros((0, 2)))
    assert info["S"] == pytest.approx(b) and info["M"] == n
    lab = info["label"]
    for j in range(by):
        for i in range(bx):
            k = j * bx + i
            assert np.all(lab[j * b:(j + 1) * b, i * b:(i + 1) * b] == k)
            np.testing.assert_allclose(params[0:2, k], [(i + 0.5) * b, (j + 0.5) * b], atol=1e-12)
            np.testing.assert_allclose(params[2:5, k], [b / math.sqrt(3), 0.0, b / math.sqrt(3)],
                                       atol=1e-12)
            np.testing.assert_array_equal(params[5:8, k], img[:, j * b, i * b].astype(np.float64))
            assert params[8, k] == pytest.approx(3 / (2 * math.pi), rel=1e-12)


def test_rectangle_segment_closed_form():
    """One seed, a w x h rectangle mask (w != h): the whole rectangle is one
    segment.  Pixel centres are uniform on w x h integer offsets, so the
    covariance is diag((w^2 - 1)/12, (h^2 - 1)/12); with + I/12 and kappa = 4:
    l1 = w / sqrt(3), l3 = h / sqrt(3), l2 = 0 (a swapped axis fails)."""
    from oracle import superpixel as sp
    W, H, w, h = 40, 30, 24, 10
    frame = np.zeros((3, H, W), np.float32)
    frame[0] = 0.3
    mask = np.zeros((H, W), bool)
    mask[5:5 + h, 3:3 + w] = True
    params, info = sp.roi_init(frame, mask, 1, 1.0, np.zeros((0, 2)))
    assert info["M"] == 1 and np.all((info["label"] >= 0) == mask)
    np.testing.assert_allclose(params[0:2, 0], [3 + w / 2, 5 + h / 2], atol=1e-12)
    np.testing.assert_allclose(params[2:5, 0], [w / math.sqrt(3), 0.0, h / math.sqrt(3)],
                               atol=1e-12)
    assert params[8, 0] == pytest.approx(w * h / (2 * math.pi * w * h / 3), rel=1e-12)


@pytest.mark.parametrize("shear", [1, -2])
def test_sheared_segment_closed_form(shear):
    """A parallelogram segment x = x0 + shear * y + t (t in [0, w), y in
    [0, h)): with Vy = (h^2 - 1)/12 and Vt = (w^2 - 1)/12 the pixel-centre
    covariance is [[shear^2 Vy + Vt, shear Vy], [shear Vy, Vy]]; Sigma =
    4 (cov + I/12), L = chol(Sigma) (Eq. 1): l2 carries the sign of the shear,
    a transposed factor or a dropped cross term fails."""
    from oracle import superpixel as sp
    w, h = 12, 9
    x0 = 30
    W, H = 80, h + 6
    frame = np.full((3, H, W), 0.5, np.float32)
    label = np.full((H, W), -1, np.int64)
    for y in range(h):
        label[3 + y, x0 + shear * y:x0 + shear * y + w] = 0
    params = sp.gaussians_from_segments(frame, label, np.array([[40.0, 7.0]]), 10.0)
    Vy, Vt = (h * h - 1) / 12.0, (w * w - 1) / 12.0
    sxx = 4 * (shear * shear * Vy + Vt + 1 / 12)
    sxy = 4 * shear * Vy
    syy = 4 * (Vy + 1 / 12)
    l1 = math.sqrt(sxx)
    l2 = sxy / l1
    l3 = math.sqrt(syy - l2 * l2)
    np.testing.assert_allclose(params[2:5, 0], [l1, l2, l3], rtol=1e-12)
    ym = 3 + h / 2
    xm = x0 + shear * (h - 1) / 2 + w / 2
    np.testing.assert_allclose(params[0:2, 0], [xm, ym], atol=1e-12)
    assert params[8, 0] == pytest.approx(w * h / (2 * math.pi * l1 * l3), rel=1e-12)


def test_mean_colour_is_exact_for_fractional_colours():
    """Colours that no fixed-point grid holds (1/3, 0.1, random floats): the
    Gaussian's colour is the plain mean of the segment's pixels."""
    from oracle import superpixel as sp
    g = rng(7)
    W = H = 12
    frame = g.uniform(0.0, 1.0, (3, H, W)).astype(np.float32)
    frame[:, :, :6] = np.float32(1.0 / 3.0)
    mask = np.ones((H, W), bool)
    S, sxy, label, _ = sp.segment(frame, mask, 4)
    params = sp.gaussians_from_segments(frame, label, sxy, S)
    for c in range(len(sxy)):
        sel = label == c
        if sel.any():
            exact = [math.fsum(float(v) for v in frame[ch][sel]) / sel.sum() for ch in range(3)]
            np.testing.assert_allclose(params[5:8, c], exact, rtol=0, atol=1e-15)


def test_assignment_exact_tie_takes_lower_index_and_gap_is_reported():
    """A pixel at exactly the same distance from two centres (same colour,
    mirror positions) joins the lower index; assign reports d1 == d2 there and
    a positive gap elsewhere."""
    from oracle import superpixel as sp
    W, H = 8, 4
    frame = np.full((3, H, W), 0.25, np.float32)
    mask = np.ones((H, W), bool)
    S, sxy, cells = sp.seeds(mask, 2)
    assert len(sxy) == 2
    col = np.full((2, 3), 0.25)
    cxy = np.array([[2.5, 2.0], [5.5, 2.0]])     # pixel x = 3 (centre 3.5) and x = 4 (4.5)
    lab, d1, d2 = sp.assign(frame, mask, col, cxy, cells, S, with_gap=True)
    # x = 3.5 and 4.5 are 1 px from one centre and 2 px from the other;
    # a centre pair at 2.5 / 6.5 would tie at x = 4.5: build that one too
    cxy_tie = np.array([[2.5, 2.0], [6.5, 2.0]])
    lab_t, d1_t, d2_t = sp.assign(frame, mask, col, cxy_tie, cells, S, with_gap=True)
    assert np.all(lab_t[:, 4] == 0)               # x centre 4.5: tie -> lower index
    assert np.all(d1_t[:, 4] == d2_t[:, 4])
    assert np.all(lab[:, 3] == 0) and np.all(lab[:, 4] == 1)
    assert np.all(d2[:, 3] > d1[:, 3])


def test_segmentation_properties_on_a_frame():
    """Every ROI pixel is labelled, nothing else; centres stay within S of
    their seeds; a pixel's segment centre (the one the last assignment used)
    is within S of it on both axes."""
    from oracle import superpixel as sp
    frame, mask = conferencing_frame(160, 120, seed=3)
    S, sxy, label, (ccol, cxy) = sp.segment(frame, mask, 200)
    assert np.all((label >= 0) == mask)
    assert np.all(np.abs(cxy - sxy) <= S + 1e-12)
    assert len(np.unique(label[label >= 0])) > 0.8 * len(sxy)
    ys, xs = np.nonzero(mask)
    lab = label[ys, xs]
    assert np.all(np.abs(xs + 0.5 - cxy[lab, 0]) <= S)
    assert np.all(np.abs(ys + 0.5 - cxy[lab, 1]) <= S)
    # brute force over all centres on a sample of pixels: the scanned 5 x 5
    # cells hold every candidate within S, so the chosen centre is the global
    # minimum of D among centres within S
    lam = (0.2 / S) ** 2
    for k in range(0, len(xs), 97):
        x, y = xs[k] + 0.5, ys[k] + 0.5
        within = (np.abs(cxy[:, 0] - x) <= S) & (np.abs(cxy[:, 1] - y) <= S)
        d = (np.sum((frame[:, ys[k], xs[k]][None, :].astype(np.float64) - ccol) ** 2, 1)
             + lam * ((cxy[:, 0] - x) ** 2 + (cxy[:, 1] - y) ** 2))
        d[~within] = np.inf
        assert lab[k] == int(np.argmin(d))


def test_background_gaussians_and_counts():
    from oracle import superpixel as sp
    frame, mask = conferencing_frame(160, 120, seed=3)
    g = rng(5)
    n = 300
    bg_xy = np.stack([g.uniform(0, 160, n), g.uniform(0, 120, n)], axis=1)
    params, info = sp.roi_init(frame, mask, n, 0.7, bg_xy)
    M = info["M"]
    assert params.shape == (9, n) and abs(M - 210) <= 20
    bg = params[:, M:]
    np.testing.assert_array_equal(bg[0:2], bg_xy[:n - M].T)
    a = (~mask).sum() / (n - M)
    np.testing.assert_allclose(bg[2], math.sqrt(4 * a / (2 * math.pi)))
    assert np.all(bg[3] == 0) and np.all(bg[8] == 0.25)


def test_tiny_roi_one_superpixel_per_pixel():
    """More superpixels asked for than the ROI has pixels: the seed step is one
    pixel, every ROI pixel is its own segment, centred on the pixel."""
    from oracle import superpixel as sp
    frame, _ = conferencing_frame(40, 30, seed=9)
    mask = np.zeros((30, 40), bool)
    mask[10:13, 20:24] = True                      # 12 pixels
    params, info = sp.roi_init(frame, mask, 100, 0.5, np.zeros((100, 2)))
    assert info["S"] == 1.0 and info["M"] == 12
    ys, xs = np.nonzero(mask)
    np.testing.assert_array_equal(params[0, :12], xs + 0.5)
    np.testing.assert_array_equal(params[1, :12], ys + 0.5)
    # a single pixel: Sigma = 4 (0 + I/12), L = diag(1/sqrt(3)), w = 1 / (2 pi / 3)
    np.testing.assert_allclose(params[2, :12], 1 / math.sqrt(3), rtol=1e-15)
    np.testing.assert_allclose(params[8, :12], 3 / (2 * math.pi), rtol=1e-15)
