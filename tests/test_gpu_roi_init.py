"""Region-of-interest superpixel initialiser on the GPU (gs2d_roi_init) against
the oracle.  Both sides decide the assignment in single precision with the
same rounded operations and form every segment sum exactly in integers, so
the Gaussians agree bit for bit (after the final rounding to float32)."""

import numpy as np
import pytest

from gs2d_inputs import background_positions, block_image, conferencing_frame

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    import paper_2505_09324_gb300 as pkg
    return pkg


def run_both(gs, frame, mask, n, roi_frac, seed):
    from oracle import superpixel as sp
    bg = background_positions(mask, n, seed=seed)
    ref, info = sp.roi_init(frame, mask, n, roi_frac, bg.T.astype(np.float64))
    got, n_roi = gs.roi_init(torch.from_numpy(frame).cuda(),
                             torch.from_numpy(mask.astype(np.uint8)).cuda(), n, roi_frac,
                             torch.from_numpy(np.ascontiguousarray(bg)).cuda())
    torch.cuda.synchronize()
    return got.cpu().numpy(), ref.astype(np.float32), n_roi, info["M"]


def test_block_image_bit_exact(gs):
    img, _ = block_image(8, 6, 6)
    mask = np.ones(img.shape[1:], bool)
    got, ref, n_roi, M = run_both(gs, img, mask, 48, 1.0, seed=1)
    assert n_roi == M == 48
    np.testing.assert_array_equal(got, ref)


def test_conferencing_frame_bit_exact(gs):
    frame, mask = conferencing_frame(320, 180, seed=3)
    got, ref, n_roi, M = run_both(gs, frame, mask, 600, 0.7, seed=4)
    assert n_roi == M
    np.testing.assert_array_equal(got, ref)


def test_full_size_1080p_bit_exact(gs):
    frame, mask = conferencing_frame(1920, 1080, seed=1)
    got, ref, n_roi, M = run_both(gs, frame, mask, 20000, 0.7, seed=11)
    assert n_roi == M and abs(M - 14000) < 100
    np.testing.assert_array_equal(got, ref)


def test_empty_mask_and_all_mask(gs):
    frame, _ = conferencing_frame(64, 48, seed=2)
    for mask in (np.zeros((48, 64), bool), np.ones((48, 64), bool)):
        got, ref, n_roi, M = run_both(gs, frame, mask, 50, 0.7, seed=5)
        assert n_roi == M
        np.testing.assert_array_equal(got, ref)


def test_large_segments_bit_exact(gs):
    """Few, large segments (S of about 180 px): the exact sums stay exact."""
    frame, mask = conferencing_frame(640, 360, seed=6)
    got, ref, n_roi, M = run_both(gs, frame, mask, 3, 0.7, seed=7)
    assert n_roi == M
    np.testing.assert_array_equal(got, ref)


def test_tiny_roi_bit_exact(gs):
    """More region Gaussians wanted than the mask has pixels: one per pixel."""
    frame, _ = conferencing_frame(40, 30, seed=9)
    mask = np.zeros((30, 40), bool)
    mask[10:13, 20:24] = True
    got, ref, n_roi, M = run_both(gs, frame, mask, 100, 0.5, seed=3)
    assert n_roi == M == 12
    np.testing.assert_array_equal(got, ref)
