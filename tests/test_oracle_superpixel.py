"""Pins for the oracle's region-of-interest superpixel initialiser (Sec. 3.2 A:
superpixel centre -> mean, segment covariance -> Cholesky factor, mean colour
-> colour)."""

import math

import numpy as np
import pytest

from gs2d_inputs import block_image, conferencing_frame, rng


def test_block_image_segments_are_the_blocks():
    """Constant-colour b x b blocks, seed step S = b: each block is a segment;
    its Gaussian has mean = block centre, Sigma = 4 (b^2/12) I (kappa = 4 times
    the second moment of a b x b square), colour = block colour and weight
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
            np.testing.assert_allclose(params[5:8, k], cols[k], atol=1e-6)
            assert params[8, k] == pytest.approx(3 / (2 * math.pi), rel=1e-12)


def test_segmentation_properties_on_a_frame():
    from oracle import superpixel as sp
    frame, mask = conferencing_frame(160, 120, seed=3)
    S, sxy, label, (ccol, cxy) = sp.segment(frame, mask, 200)
    assert np.all((label >= 0) == mask)                  # every ROI pixel, nothing else
    assert np.all(np.abs(cxy - sxy) <= S + 1e-12)        # the leash
    assert len(np.unique(label[label >= 0])) > 0.8 * len(sxy)
    # a pixel's centre is within S (per axis) of the centre of its segment
    # as used by the last assignment: recompute the previous centres
    h, w = mask.shape
    ys, xs = np.nonzero(mask)
    # segment Gaussians: Sigma equals the covariance of the pixel centres + I/12
    params = sp.gaussians_from_segments(frame, label, sxy, S)
    for k in np.unique(label[label >= 0])[:20]:
        sel = label == k
        pts = np.stack([xs[sel[ys, xs]] + 0.5, ys[sel[ys, xs]] + 0.5])
        cov = 4 * (np.cov(pts, bias=True) + np.eye(2) / 12)
        Lm = np.array([[params[2, k], 0], [params[3, k], params[4, k]]])
        np.testing.assert_allclose(Lm @ Lm.T, cov, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(params[0:2, k], pts.mean(axis=1), rtol=0, atol=1e-9)
        np.testing.assert_allclose(params[5:8, k], frame[:, sel].mean(axis=1), atol=1e-6)


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


def test_segment_sums_are_exact_and_order_free():
    """The integer segment sums equal the plain sums of the definitions (u =
    2 x + 1 - 2 floor(q), colours rint(c 2^20)), whatever the pixel order; the
    quantised mean colour is within 2^-21 of the exact mean."""
    from oracle import superpixel as sp
    frame, mask = conferencing_frame(96, 64, seed=8)
    S, sxy, label, _ = sp.segment(frame, mask, 60)
    sm = sp.segment_sums(frame, label, sxy)
    for c in np.unique(label[label >= 0])[:15]:
        ys, xs = np.nonzero(label == c)
        fx, fy = math.floor(sxy[c, 0]), math.floor(sxy[c, 1])
        u = [2 * int(x) + 1 - 2 * fx for x in xs]
        v = [2 * int(y) + 1 - 2 * fy for y in ys]
        assert sm["n"][c] == len(xs)
        assert (sm["u"][c], sm["v"][c]) == (sum(u), sum(v))
        assert sm["uu"][c] == sum(a * a for a in u) and sm["uv"][c] == sum(
            a * b for a, b in zip(u, v))
        for ch, key in enumerate("rgb"):
            q = [int(np.rint(float(frame[ch, y, x]) * 2.0 ** 20)) for y, x in zip(ys, xs)]
            assert sm[key][c] == sum(q)
            exact = float(np.mean(frame[ch, ys, xs].astype(np.float64)))
            assert abs(sm[key][c] / (len(xs) * 2.0 ** 20) - exact) <= 2.0 ** -21 + 1e-15


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
