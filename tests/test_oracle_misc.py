"""Pins for the oracle's Adam step (against torch.optim.Adam on CPU, the library
special case), loss and PSNR (closed forms), and the input generators."""

import math

import numpy as np
import pytest

from gs2d_inputs import conferencing_frame, random_gaussians, smooth_noise_target


def test_adam_matches_torch_cpu(oracle):
    torch = pytest.importorskip("torch")
    g = np.random.Generator(np.random.PCG64(5))
    p0 = g.normal(size=(9, 17))
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for step in range(1, 8):
        grad = g.normal(size=p0.shape) * (10.0 ** g.uniform(-4, 1))
        opt.zero_grad()
        tp.grad = torch.tensor(grad, dtype=torch.float64)
        opt.step()
        p, m, v = oracle.adam_step(p, grad, m, v, step)
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_loss_and_psnr_closed_forms(oracle):
    t = np.full((3, 8, 8), 0.5)
    img = t + 0.1
    loss, g = oracle.l2_loss(img, t)
    assert loss == pytest.approx(0.01, rel=1e-12)
    np.testing.assert_allclose(g, 2 * 0.1 / img.size)
    assert oracle.psnr(img, t) == pytest.approx(20.0, rel=1e-12)
    # PSNR clamps the rendered image to [0, 1]; the loss does not
    assert oracle.psnr(np.full_like(t, 7.0), np.ones_like(t)) == math.inf
    assert oracle.l2_loss(np.full_like(t, 7.0), np.ones_like(t))[0] == pytest.approx(36.0)


def test_generators_are_seeded_and_shaped():
    a = random_gaussians(100, 256, 256, seed=0)
    b = random_gaussians(100, 256, 256, seed=0)
    assert a.shape == (9, 100) and a.dtype == np.float32
    np.testing.assert_array_equal(a, b)
    assert np.all((a[0] >= 0) & (a[0] < 256))
    assert np.all((a[2] >= 1) & (a[2] <= 8)) and np.all((a[8] >= 0.2) & (a[8] <= 1))
    t = smooth_noise_target(64, 48, seed=1)
    assert t.shape == (3, 48, 64) and t.min() >= 0 and t.max() <= 1
    f, m = conferencing_frame(320, 180, seed=1)
    assert f.shape == (3, 180, 320) and m.shape == (180, 320)
    assert abs(m.mean() - 0.3) < 0.01


def test_contributes_matches_single_gaussian_renders(oracle):
    """The per-pair predicate against the oracle's renderer: a Gaussian
    contributes at a pixel exactly when its render alone is non-zero there."""
    import numpy as np
    from gs2d_inputs import random_gaussians
    W, H = 40, 30
    p = random_gaussians(12, W, H, seed=4).astype(np.float64)
    p[8, 3] = 0.001          # invisible (|w| < 1/255)
    p[2, 5] = 1e-5           # degenerate
    g = np.random.Generator(np.random.PCG64(5))
    xy = np.stack([g.integers(0, W, 300), g.integers(0, H, 300)], axis=1)
    definite, ambiguous = oracle.contributes(p, xy)
    for i in range(p.shape[1]):
        single = p[:, i:i + 1].copy()
        single[5:8] = 1.0        # a non-zero colour shows every contribution
        vals = oracle.render_pixels(single, xy)[0]
        nz = vals != 0.0
        sure = ~ambiguous[:, i]
        assert np.array_equal(nz[sure], definite[sure, i]), i
    assert not definite[:, 3].any() and not definite[:, 5].any()


def test_subject_moves_rigidly():
    """The subject's texture lives in object coordinates: a translation by
    whole pixels shifts the interior of the subject exactly (the recipe's
    rigid motion, no resampling)."""
    from gs2d_inputs import SubjectMotion
    W, H = 200, 120
    mo = SubjectMotion(v=3.0, direction=0.0, omega=0.0)
    f0, m0 = conferencing_frame(W, H, seed=4, t=0, motion=mo)
    f2, m2 = conferencing_frame(W, H, seed=4, t=2, motion=mo)   # 6 px to the right
    inner = np.zeros_like(m0)
    inner[:, 6:] = m0[:, :-6] & m2[:, 6:]
    # away from the soft edge on both frames
    from scipy.ndimage import binary_erosion
    inner = binary_erosion(inner, iterations=4)
    assert inner.sum() > 1000
    ys, xs = np.nonzero(inner)
    np.testing.assert_allclose(f2[:, ys, xs], f0[:, ys, xs - 6], atol=2e-6)


def test_clip_table_and_background_positions_follow_the_recipe():
    from gs2d_inputs import background_positions, clip_table
    t = clip_table(64, 7)
    assert t == clip_table(64, 7)
    assert {(c["width"], c["height"]) for c in t} <= {(640, 360), (1280, 720), (1920, 1080)}
    assert all(2000 <= c["n"] <= 50000 for c in t)
    ns = np.log([c["n"] for c in t])
    assert ns.min() < np.log(6000) and ns.max() > np.log(20000)  # spread over the log range
    _, mask = conferencing_frame(160, 96, seed=2)
    xy = background_positions(mask, 500, seed=3)
    assert xy.shape == (2, 500)
    xi, yi = np.floor(xy[0]).astype(int), np.floor(xy[1]).astype(int)
    assert not mask[yi, xi].any()  # every position on a background pixel
