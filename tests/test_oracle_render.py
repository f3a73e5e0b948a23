"""Pins for the oracle's forward render (Eq. 2 with the factorised covariance of
Eq. 1, Sec. 3.1).  Each test checks the oracle against something other than
itself: closed forms, lattice-sum identities, exact symmetries."""

import math

import numpy as np
import pytest

from gs2d_inputs import random_gaussians

pytestmark = pytest.mark.filterwarnings("ignore")


def one(mx, my, l1, l2, l3, c=(0.2, 0.5, 0.9), w=0.7):
    return np.array([[mx], [my], [l1], [l2], [l3], [c[0]], [c[1]], [c[2]], [w]], np.float64)


def test_peak_equals_weighted_colour(oracle):
    # A Gaussian centred on a pixel centre has sigma = 0 there, so C = w * c exactly.
    p = one(20.5, 30.5, 3.0, 0.0, 3.0)
    img = oracle.render(p, 48, 48)
    np.testing.assert_array_equal(img[:, 30, 20], 0.7 * np.array([0.2, 0.5, 0.9]))
    # the peak is the maximum of every channel
    assert np.all(img[:, 30, 20] == img.reshape(3, -1).max(axis=1))


def test_lattice_moments_recover_mean_and_covariance(oracle):
    """With the cut-off disabled, lattice sums of a well-sampled Gaussian equal
    its integrals (Poisson summation; aliasing ~exp(-2 pi^2 lambda_min) ~ 0):
    mass = w c 2 pi sqrt(det Sigma), first moment = mu, second = Sigma = L L^T."""
    cfg = oracle.Config(sigma_cut=60.0, alpha_min=1e-30)
    l1, l2, l3 = 2.5, 1.2, 3.0
    mx, my = 63.37, 58.91
    p = one(mx, my, l1, l2, l3, c=(1.0, 0.5, 0.25), w=0.8)
    W = H = 128
    img = oracle.render(p, W, H, cfg, fast=True)
    sigma = np.array([[l1 * l1, l1 * l2], [l1 * l2, l2 * l2 + l3 * l3]])
    mass_expected = 0.8 * 2 * math.pi * math.sqrt(np.linalg.det(sigma))
    f = img[0]
    mass = f.sum()
    assert abs(mass - mass_expected) <= 1e-10 * mass_expected
    np.testing.assert_allclose(img[1].sum(), 0.5 * mass_expected, rtol=1e-10)
    xs = np.arange(W) + 0.5
    ys = np.arange(H) + 0.5
    X, Y = np.meshgrid(xs, ys)
    m1 = np.array([(f * X).sum(), (f * Y).sum()]) / mass
    np.testing.assert_allclose(m1, [mx, my], rtol=0, atol=1e-9)
    dx, dy = X - mx, Y - my
    cov = np.array([[(f * dx * dx).sum(), (f * dx * dy).sum()],
                    [(f * dx * dy).sum(), (f * dy * dy).sum()]]) / mass
    np.testing.assert_allclose(cov, sigma, rtol=1e-9, atol=1e-9)
    # the transposed factorisation L^T L would give a different covariance
    wrong = np.array([[l1 * l1 + l2 * l2, l2 * l3], [l2 * l3, l3 * l3]])
    assert np.abs(cov - wrong).max() > 0.5


@pytest.mark.parametrize("s", [4.0, 8.0])
def test_truncated_integral_closed_form(oracle, s):
    """Truncation at sigma <= 4.5: mass -> w c 2 pi s^2 (1 - e^{-4.5}); the
    lattice-count error at the cut is O(e^{-4.5} R^{2/3}) relative to the mass."""
    p = one(64.5, 64.5, s, 0.0, s, c=(1.0, 1.0, 1.0), w=1.0)
    img = oracle.render(p, 129, 129)
    expected = 2 * math.pi * s * s * (1 - math.exp(-4.5))
    assert abs(img[0].sum() - expected) / expected < 3e-3


def test_truncation_exact_integer_offsets(oracle):
    """Centred on a pixel centre, offsets are integers (i, j): the render must
    equal the sum over integer offsets with (i^2 + j^2) / (2 s^2) <= tau of
    w c exp(-(i^2 + j^2)/(2 s^2)), tau = min(4.5, ln(255 |w|))."""
    s = 3.0
    for w in (1.0, 0.02, -0.5):
        tau = min(4.5, math.log(255 * abs(w)))
        p = one(32.5, 32.5, s, 0.0, s, c=(1.0, 1.0, 1.0), w=w)
        img, lo, hi = oracle.render(p, 65, 65, ambiguity=True)
        total = 0.0
        count = 0
        for i in range(-20, 21):
            for j in range(-20, 21):
                q = (i * i + j * j) / (2 * s * s)
                if q <= tau:
                    total += w * math.exp(-q)
                    count += 1
        # points exactly on the cut (i^2 + j^2 = 81 for tau = 4.5) sit in the
        # ambiguity band: definite + band = the inclusive sum
        full = img[0] + lo[0] + hi[0]
        assert abs(full.sum() - total) <= 1e-12 * abs(total)
        assert np.count_nonzero(full) == count


def test_weight_below_alpha_min_contributes_nothing(oracle):
    p = one(10.5, 10.5, 2.0, 0.0, 2.0, w=0.5 / 255)
    assert not np.any(oracle.render(p, 24, 24))


def test_degenerate_and_nonfinite_are_culled(oracle):
    cases = [one(10.5, 10.5, 1e-5, 0.0, 1e-5), one(np.nan, 10.5, 2, 0, 2),
             one(10.5, 10.5, 2, np.inf, 2), one(10.5, 10.5, 2, 0, 2, c=(np.nan, 0, 0)),
             one(10.5, 10.5, 2, 0, 2, w=0.0)]
    for p in cases:
        assert not np.any(oracle.render(p, 24, 24))
    assert not np.any(oracle.render(np.zeros((9, 0)), 24, 24))


def test_tile_translation_is_exact(oracle):
    """Shifting every mean by whole tiles on a larger canvas shifts the image
    bit-exactly (means on a dyadic grid keep p - mu exact)."""
    p = random_gaussians(40, 64, 48, seed=3).astype(np.float64)
    p[0:2] = np.round(p[0:2] * 256) / 256
    a = oracle.render(p, 64, 48)
    q = p.copy()
    q[0] += 32
    q[1] += 16
    b = oracle.render(q, 128, 96)
    # compare where no Gaussian from outside the original canvas can reach
    np.testing.assert_array_equal(b[:, 16:16 + 48, 32:32 + 64][:, 12:-12, 12:-12],
                                  a[:, 12:-12, 12:-12])


def test_mirror_symmetry(oracle):
    """x -> W - x maps Sigma_xy -> -Sigma_xy, i.e. l2 -> -l2 (Eq. 1)."""
    W, H = 64, 40
    p = random_gaussians(30, W, H, seed=5).astype(np.float64)
    a = oracle.render(p, W, H)
    q = p.copy()
    q[0] = W - p[0]
    q[3] = -p[3]
    b = oracle.render(q, W, H)
    np.testing.assert_allclose(b[:, :, ::-1], a, rtol=0, atol=1e-12)


def test_colour_linearity_and_permutation(oracle):
    W, H = 50, 37
    p = random_gaussians(60, W, H, seed=7).astype(np.float64)
    a = oracle.render(p, W, H)
    q = p.copy()
    q[5:8] *= 2
    np.testing.assert_array_equal(oracle.render(q, W, H), 2 * a)
    perm = np.random.Generator(np.random.PCG64(1)).permutation(p.shape[1])
    np.testing.assert_allclose(oracle.render(p[:, perm], W, H), a, rtol=0, atol=1e-12)


def test_fast_mode_equals_brute_force(oracle):
    W, H = 100, 70
    p = random_gaussians(300, W, H, seed=11)
    a = oracle.render(p, W, H, fast=False)
    b = oracle.render(p, W, H, fast=True)
    np.testing.assert_array_equal(a, b)


def test_render_pixels_matches_full_render(oracle):
    W, H = 64, 48
    p = random_gaussians(80, W, H, seed=13)
    img, lo, hi = oracle.render(p, W, H, ambiguity=True)
    xy = np.array([[0, 0], [63, 47], [10, 20], [31, 7]])
    v, vlo, vhi = oracle.render_pixels(p, xy, ambiguity=True)
    for k, (x, y) in enumerate(xy):
        np.testing.assert_allclose(v[:, k], img[:, y, x], rtol=0, atol=1e-13)
        np.testing.assert_allclose(vlo[:, k], lo[:, y, x], rtol=0, atol=1e-13)
        np.testing.assert_allclose(vhi[:, k], hi[:, y, x], rtol=0, atol=1e-13)


def test_ambiguity_band_brackets_either_choice(oracle):
    """A pixel placed exactly on the cut-off ellipse is ambiguous: the definite
    image excludes it, and [lo, hi] spans its contribution."""
    s = 2.0
    # offset (6, 0): sigma = 36 / 8 = 4.5 = sigma_cut
    p = one(10.5, 10.5, s, 0.0, s, c=(1.0, 1.0, 1.0), w=1.0)
    img, lo, hi = oracle.render(p, 24, 24, ambiguity=True)
    assert img[0, 10, 16] == 0.0
    assert hi[0, 10, 16] == pytest.approx(math.exp(-4.5), rel=1e-12)
    assert lo[0, 10, 16] == 0.0
