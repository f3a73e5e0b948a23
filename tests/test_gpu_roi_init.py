"""Region-of-interest superpixel initialiser on the GPU (gs2d_roi_init, Sec.
3.2 A) against the plain double-precision oracle, one K-means iteration at a
time.

The GPU decides its assignments in FP32 and forms segment sums in exact
integers (pixel centres as 2x + 1 - 2 floor(seed), colours quantised to
2^-20); the oracle computes the definition in float64.  So the check is made
step by step from shared states (gs2d_roi_init_trace writes out every
iteration's centres and labels):

* labels: given the GPU's centres of iteration k, the oracle's labels equal the
  GPU's except at near-tie pixels -- where the GPU's pick lies within the
  FP32 rounding band of the best float64 distance, |D_gpu - D_best| <=
  2^-20 (D_best + D_second) (an FP32 evaluation of D has relative error
  below 7 * 2^-24 per candidate), or where a candidate sits on the edge of the
  S-window to within FP32 rounding (|S - max(|dx|, |dy|)| <= 4e-7 S + 1e-6);
* centres: given the GPU's labels of iteration k, the oracle's update equals
  the GPU's centres of iteration k + 1 within one float32 ulp (positions: the
  exact mean rounded once to float32) and 2^-21 + one ulp (colours: the
  2^-20 quantisation moves a mean by at most 2^-21);
* Gaussians: from the GPU's final labels, the oracle's Gaussians equal the
  GPU's within one float32 ulp (means), 4 ulp relative (Cholesky factor and
  weight: a few double operations, then one rounding) and 2^-21 + one ulp
  (colours)."""

import numpy as np
import pytest

from gs2d_inputs import background_positions, block_image, conferencing_frame

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ULP = 2.0 ** -23
COLOUR_Q = 2.0 ** -21


@pytest.fixture(scope="module")
def gs():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    import paper_2505_09324_gb300 as pkg
    return pkg


def gpu_trace(gs, frame, mask, n, roi_frac, seed):
    bg = background_positions(mask, n, seed=seed)
    params, n_roi, cen, lab = gs.roi_init_trace(
        torch.from_numpy(frame).cuda(), torch.from_numpy(mask.astype(np.uint8)).cuda(), n,
        roi_frac, torch.from_numpy(np.ascontiguousarray(bg)).cuda())
    torch.cuda.synchronize()
    return params.cpu().numpy(), n_roi, cen.cpu().numpy(), lab.cpu().numpy(), bg


def check_labels(sp, frame, mask, ccol, cxy, cells, S, gl):
    """Oracle labels from the GPU's centres against the GPU's labels; returns
    the number of near-tie pixels where they differ."""
    lab, d1, d2 = sp.assign(frame, mask, ccol, cxy, cells, S, with_gap=True)
    diff = np.nonzero(lab != gl)
    if len(diff[0]) == 0:
        return 0
    ys, xs = diff
    assert np.all(mask[ys, xs]), "labels differ outside the mask"
    lam = (0.2 / S) ** 2
    for y, x in zip(ys, xs):
        g, o = int(gl[y, x]), int(lab[y, x])
        px, py = x + 0.5, y + 0.5

        def dist(c):
            dx, dy = px - cxy[c, 0], py - cxy[c, 1]
            dc = np.sum((frame[:, y, x].astype(np.float64) - ccol[c]) ** 2)
            return dc + lam * (dx * dx + dy * dy), S - max(abs(dx), abs(dy))

        edge = 4e-7 * S + 1e-6
        ok = False
        if g >= 0:
            dg, mg = dist(g)
            ok = abs(mg) <= edge or (mg >= 0 and dg - d1[y, x] <= 2.0 ** -20 * (d1[y, x] + d2[y, x]))
        if not ok and o >= 0:
            ok = abs(dist(o)[1]) <= edge
        assert ok, f"pixel ({x}, {y}): GPU centre {g}, oracle centre {o}"
    return len(ys)


def check_step_by_step(gs, frame, mask, n, roi_frac, seed, iterations=range(10)):
    from oracle import superpixel as sp
    params, n_roi, cen, lab, bg = gpu_trace(gs, frame, mask, n, roi_frac, seed)
    S, sxy, cells = sp.seeds(mask, int(round(roi_frac * n)), max_seeds=n)
    M = len(sxy)
    assert n_roi == M
    # iteration 0: the seeds, with the frame's colour at the seed's pixel
    col0, xy0 = sp.initial_centres(frame, sxy)
    np.testing.assert_array_equal(cen[0, 3:5, :M].T, xy0.astype(np.float32))
    np.testing.assert_array_equal(cen[0, 0:3, :M].T, col0.astype(np.float32))
    near = 0
    for k in iterations:
        ccol = cen[k, 0:3, :M].T.astype(np.float64)
        cxy = cen[k, 3:5, :M].T.astype(np.float64)
        near += check_labels(sp, frame, mask, ccol, cxy, cells, S, lab[k])
        if k + 1 < 10:
            ncol, nxy = sp.update(frame, lab[k].astype(np.int64), ccol, cxy, sxy, S)
            gxy = cen[k + 1, 3:5, :M].T.astype(np.float64)
            gcol = cen[k + 1, 0:3, :M].T.astype(np.float64)
            assert np.all(np.abs(gxy - nxy) <= ULP * np.abs(nxy) + 1e-12)
            assert np.all(np.abs(gcol - ncol) <= COLOUR_Q + ULP * np.abs(ncol))
    # the Gaussians from the GPU's final labels
    ref = sp.gaussians_from_segments(frame, lab[9].astype(np.int64), sxy, S)
    got = params[:, :M].astype(np.float64)
    assert np.all(np.abs(got[0:2] - ref[0:2]) <= ULP * np.abs(ref[0:2]) + 1e-12)
    scale = np.maximum(np.abs(ref[2]), np.abs(ref[4]))
    assert np.all(np.abs(got[2:5] - ref[2:5]) <= 4 * ULP * scale + 1e-12)
    assert np.all(np.abs(got[5:8] - ref[5:8]) <= COLOUR_Q + ULP * np.abs(ref[5:8]))
    assert np.all(np.abs(got[8] - ref[8]) <= 4 * ULP * np.abs(ref[8]))
    # the background Gaussians
    bg_ref = sp.background_gaussians(frame, mask, bg.T.astype(np.float64), n - M)
    assert np.all(np.abs(params[:, M:] - bg_ref) <= ULP * np.abs(bg_ref) + 1e-12)
    return M, near


def test_block_image_is_the_oracle_exactly(gs):
    """No near-ties and no fractional means: labels equal at every iteration,
    the Gaussians equal the closed form of the blocks."""
    img, _ = block_image(8, 6, 6)
    mask = np.ones(img.shape[1:], bool)
    M, near = check_step_by_step(gs, img, mask, 48, 1.0, seed=1)
    assert M == 48 and near == 0


def test_conferencing_frame_step_by_step(gs):
    frame, mask = conferencing_frame(320, 180, seed=3)
    M, near = check_step_by_step(gs, frame, mask, 600, 0.7, seed=4)
    assert M > 0


def test_full_size_1080p_step_by_step(gs):
    """The benchmark's frame: every iteration's labels, a sample of updates
    (the first, a middle and the last), the final Gaussians."""
    frame, mask = conferencing_frame(1920, 1080, seed=1)
    M, near = check_step_by_step(gs, frame, mask, 20000, 0.7, seed=11, iterations=(0, 4, 9))
    assert abs(M - 14000) < 100


def test_empty_mask_and_all_mask(gs):
    frame, _ = conferencing_frame(64, 48, seed=2)
    for mask in (np.zeros((48, 64), bool), np.ones((48, 64), bool)):
        check_step_by_step(gs, frame, mask, 50, 0.7, seed=5)


def test_large_segments(gs):
    """Few, large segments (S of about 180 px)."""
    frame, mask = conferencing_frame(640, 360, seed=6)
    check_step_by_step(gs, frame, mask, 3, 0.7, seed=7)


def test_tiny_roi_one_superpixel_per_pixel(gs):
    """More region Gaussians wanted than the mask has pixels: one per pixel."""
    frame, _ = conferencing_frame(40, 30, seed=9)
    mask = np.zeros((30, 40), bool)
    mask[10:13, 20:24] = True
    M, near = check_step_by_step(gs, frame, mask, 100, 0.5, seed=3)
    assert M == 12 and near == 0


def test_roi_init_equals_its_trace(gs):
    """gs2d_roi_init and gs2d_roi_init_trace give the same Gaussians bit for
    bit (the trace only copies states out)."""
    frame, mask = conferencing_frame(320, 180, seed=3)
    bg = torch.from_numpy(background_positions(mask, 600, seed=4)).cuda()
    f = torch.from_numpy(frame).cuda()
    m = torch.from_numpy(mask.astype(np.uint8)).cuda()
    a, na = gs.roi_init(f, m, 600, 0.7, bg)
    b, nb, _, _ = gs.roi_init_trace(f, m, 600, 0.7, bg)
    assert na == nb
    assert torch.equal(a, b)
