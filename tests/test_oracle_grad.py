"""Pins for the oracle's analytic gradients through Eq. 2 and Eq. 1 (Sec. 3.1:
the method optimises the Cholesky factors by gradient descent).  The analytic
gradient is checked against central finite differences of the oracle's own
double-precision loss, on tiny inputs chosen so that no pixel sits near the
cut-off (where the loss is discontinuous), and against exact symmetries."""

import math

import numpy as np
import pytest

from gs2d_inputs import random_gaussians, smooth_noise_target


def loss_of(oracle, p, target, cfg):
    img = oracle.render(p, target.shape[2], target.shape[1], cfg)
    return oracle.l2_loss(img, target)[0]


def clean_case(oracle, W, H, n, seed, cfg):
    """Seeded case with no pair inside a wide band around the cut-off."""
    wide = oracle.Config(sigma_cut=cfg.sigma_cut, alpha_min=cfg.alpha_min, amb_tol=5e-3)
    for s in range(seed, seed + 200):
        p = random_gaussians(n, W, H, seed=s).astype(np.float64)
        _, lo, hi = oracle.render(p, W, H, wide, ambiguity=True)
        if not np.any(lo) and not np.any(hi):
            return p
    raise RuntimeError("no clean case found")


@pytest.mark.parametrize("seed", [100, 300])
def test_gradient_matches_central_differences(oracle, seed):
    cfg = oracle.Config()
    W, H, n = 24, 20, 5
    p = clean_case(oracle, W, H, n, seed, cfg)
    target = smooth_noise_target(W, H, seed=seed + 1).astype(np.float64)
    res = oracle.loss_and_grad(p, target, cfg)
    grad = res["grad"]
    assert not np.any(res["grad_unc"])
    fd = np.zeros_like(p)
    for r in range(9):
        for i in range(n):
            h = 1e-6 * max(1.0, abs(p[r, i]))
            a = p.copy()
            a[r, i] += h
            b = p.copy()
            b[r, i] -= h
            fd[r, i] = (loss_of(oracle, a, target, cfg) - loss_of(oracle, b, target, cfg)) / (2 * h)
    scale = np.abs(fd).max(axis=1, keepdims=True)
    np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=0)  # tight where it is large
    assert np.all(np.abs(grad - fd) <= 1e-6 * np.abs(fd) + 1e-9 * scale)


def test_gradient_without_cutoff_matches_differences_with_negative_weights(oracle):
    """Cut-off disabled (sigma_cut large): the loss is smooth everywhere, so FD
    applies at any point, including negative weights and sheared factors."""
    cfg = oracle.Config(sigma_cut=40.0, alpha_min=1e-30)
    W, H, n = 20, 18, 4
    g = np.random.Generator(np.random.PCG64(9))
    p = random_gaussians(n, W, H, seed=21).astype(np.float64)
    p[3] = g.normal(0, 2.0, n)
    p[8] = g.uniform(-1, 1, n)
    target = smooth_noise_target(W, H, seed=4).astype(np.float64)
    grad = oracle.loss_and_grad(p, target, cfg)["grad"]
    fd = np.zeros_like(p)
    for r in range(9):
        for i in range(n):
            h = 1e-6 * max(1.0, abs(p[r, i]))
            a = p.copy()
            a[r, i] += h
            b = p.copy()
            b[r, i] -= h
            fd[r, i] = (loss_of(oracle, a, target, cfg) - loss_of(oracle, b, target, cfg)) / (2 * h)
    np.testing.assert_allclose(grad, fd, rtol=2e-6, atol=1e-12)


def test_symmetric_loss_has_zero_mean_and_shear_gradient(oracle):
    """Isotropic Gaussian on a pixel centre, constant target: the loss is
    invariant under reflection about mu, so dL/dmu = 0, and under x -> -x,
    which maps l2 -> -l2, so dL/dl2 = 0 at l2 = 0."""
    cfg = oracle.Config()
    p = np.array([[16.5], [12.5], [2.5], [0.0], [2.5], [0.3], [0.6], [0.9], [0.8]])
    target = np.full((3, 25, 33), 0.25)
    grad = oracle.loss_and_grad(p, target, cfg)["grad"]
    assert abs(grad[0, 0]) < 1e-15 and abs(grad[1, 0]) < 1e-15
    assert abs(grad[3, 0]) < 1e-15
    # isotropy: dL/dl1 = dL/dl3 (swap of axes) and both are non-zero
    assert grad[2, 0] == pytest.approx(grad[4, 0], rel=1e-12)
    assert abs(grad[2, 0]) > 1e-6


def test_colour_gradient_closed_form(oracle):
    """dL/dc_ch = sum_p g_ch(p) w exp(-sigma): with g = 1 everywhere and the cut
    disabled, it is w * 2 pi sqrt(det Sigma) (the lattice mass)."""
    cfg = oracle.Config(sigma_cut=60.0, alpha_min=1e-30)
    l1, l2, l3, w = 2.0, 0.7, 2.5, 0.6
    p = np.array([[40.2], [39.7], [l1], [l2], [l3], [0.3], [0.6], [0.9], [w]])
    g = np.ones((3, 80, 80))
    grad = oracle.render_grad(p, 80, 80, g, cfg, fast=True)
    expected = w * 2 * math.pi * l1 * l3
    np.testing.assert_allclose(grad[5:8, 0], expected, rtol=1e-10)
    # and dL/dw = sum_ch c_ch * 2 pi sqrt(det)
    np.testing.assert_allclose(grad[8, 0], (0.3 + 0.6 + 0.9) * 2 * math.pi * l1 * l3, rtol=1e-10)
    # translation invariance of the mass: dL/dmu = 0 for constant g
    assert abs(grad[0, 0]) < 1e-9 and abs(grad[1, 0]) < 1e-9
    # d(mass)/dl1 = mass / l1 (mass is proportional to l1 l3), dl2 = 0
    np.testing.assert_allclose(grad[2, 0], w * 1.8 * 2 * math.pi * l3, rtol=1e-9)
    assert abs(grad[3, 0]) < 1e-9


def test_subset_gradient_matches_full(oracle):
    W, H = 40, 30
    p = random_gaussians(20, W, H, seed=17)
    g = smooth_noise_target(W, H, seed=2).astype(np.float64) - 0.5
    full = oracle.render_grad(p, W, H, g)
    which = np.array([3, 7, 19])
    sub = oracle.render_grad(p, W, H, g, which=which)
    np.testing.assert_array_equal(sub[:, which], full[:, which])
    rest = np.setdiff1d(np.arange(20), which)
    assert not np.any(sub[:, rest])
