"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds only input generation (random Gaussian sets, analytic frames,
motion tracks, clip tables).  It contains none of the rasterizer's arithmetic:
no projection, binning, blending, gradients or optimiser steps.  Every generator
draws from ``numpy.random.Generator(PCG64(seed))`` so that both sides of a parity
test see identical inputs.

Parameter layout used throughout: a float32 array of shape ``[9, n]`` whose rows
are ``mu_x, mu_y, l1, l2, l3, c_r, c_g, c_b, w`` (Sec. 3.1: position, Cholesky
vector of Eq. 1, colour; ``w`` is the per-Gaussian weight folded into the
colour coefficient of Eq. 2).  Images are float32 ``[3, H, W]``, pixel ``(x, y)``
has its centre at ``(x + 0.5, y + 0.5)``.

Workload recipes (the paper's VCD talking-head data is not available; these are
stand-ins with the same structure):

* ``random_gaussians``: means uniform over the image, diagonal Cholesky entries
  log-uniform in [1, 8] px, off-diagonal N(0, 1) px, colours U[0, 1], weights
  U[0.2, 1].
* ``smooth_noise_target``: 0.5 + 0.5 * (sum of 16 random low-frequency plane
  waves, at most 4 cycles per image) / (sum of |amplitudes|), per channel.
* ``conferencing_frame``: smooth low-frequency background plus a centred
  elliptical "subject" of 30 % of the frame area (aspect 1.3, 1.5 px smoothstep
  edge) carrying band-limited texture (64 plane waves, wavelengths 24-96 px,
  total amplitude 0.15) evaluated in object coordinates, so rigid motion of the
  subject is exact.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "rng",
    "random_gaussians",
    "smooth_noise_target",
    "SubjectMotion",
    "conferencing_frame",
    "conferencing_gaussians",
    "background_positions",
    "block_image",
    "conferencing_sequence",
    "random_motion",
    "clip_table",
    "ROW_NAMES",
]

ROW_NAMES = ("mu_x", "mu_y", "l1", "l2", "l3", "c_r", "c_g", "c_b", "w")


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_gaussians(n: int, width: int, height: int, seed: int,
                     l_range=(1.0, 8.0), l2_std=1.0, w_range=(0.2, 1.0)) -> np.ndarray:
    """``[9, n]`` float32 Gaussian set drawn from the distributions listed above."""
    g = rng(seed)
    p = np.empty((9, n), dtype=np.float64)
    p[0] = g.uniform(0.0, width, n)
    p[1] = g.uniform(0.0, height, n)
    lo, hi = math.log(l_range[0]), math.log(l_range[1])
    p[2] = np.exp(g.uniform(lo, hi, n))
    p[3] = g.normal(0.0, l2_std, n)
    p[4] = np.exp(g.uniform(lo, hi, n))
    p[5:8] = g.uniform(0.0, 1.0, (3, n))
    p[8] = g.uniform(w_range[0], w_range[1], n)
    return p.astype(np.float32)


def _plane_wave_sum(width, height, kx, ky, phase, amp):
    """sum_j amp_j * sin(kx_j * x + ky_j * y + phase_j) at pixel centres.

    Evaluated separably as one matrix product: with
    sin(a + b) = sin a cos b + cos a sin b, the sum is
    [cos B | sin B] (H x 2J) times [amp sin A ; amp cos A] (2J x W).
    """
    xs = np.arange(width, dtype=np.float64) + 0.5
    ys = np.arange(height, dtype=np.float64) + 0.5
    kx, ky = np.asarray(kx, np.float64), np.asarray(ky, np.float64)
    amp, phase = np.asarray(amp, np.float64), np.asarray(phase, np.float64)
    A = np.outer(kx, xs)                       # [J, W]
    B = np.outer(ys, ky) + phase[None, :]      # [H, J]
    left = np.concatenate([np.cos(B), np.sin(B)], axis=1)                        # [H, 2J]
    right = np.concatenate([amp[:, None] * np.sin(A), amp[:, None] * np.cos(A)])  # [2J, W]
    return left @ right


def smooth_noise_target(width: int, height: int, seed: int, terms: int = 16,
                        max_cycles: int = 4) -> np.ndarray:
    """Seeded smooth-noise field, float32 ``[3, H, W]`` with values in [0, 1]."""
    g = rng(seed)
    img = np.empty((3, height, width), dtype=np.float64)
    for ch in range(3):
        cx = g.integers(-max_cycles, max_cycles + 1, terms)
        cy = g.integers(-max_cycles, max_cycles + 1, terms)
        amp = g.uniform(0.2, 1.0, terms)
        ph = g.uniform(0.0, 2.0 * math.pi, terms)
        kx = 2.0 * math.pi * cx / width
        ky = 2.0 * math.pi * cy / height
        s = _plane_wave_sum(width, height, kx, ky, ph, amp)
        img[ch] = 0.5 + 0.5 * s / np.sum(np.abs(amp))
    return img.astype(np.float32)


@dataclasses.dataclass(frozen=True)
class SubjectMotion:
    """Rigid motion of the foreground subject: translation ``v`` px/frame along
    ``direction`` (radians) and rotation ``omega`` degrees/frame."""

    v: float = 0.0
    direction: float = 0.0
    omega: float = 0.0


def random_motion(seed: int) -> SubjectMotion:
    g = rng(seed)
    return SubjectMotion(v=float(g.uniform(0.0, 4.0)), direction=float(g.uniform(0.0, 2 * math.pi)),
                         omega=float(g.uniform(0.0, 1.0)))


def _scene_spec(seed: int):
    g = rng(seed)
    bg = []
    for ch in range(3):
        cx = g.integers(-3, 4, 8)
        cy = g.integers(-3, 4, 8)
        amp = g.uniform(0.2, 1.0, 8)
        ph = g.uniform(0.0, 2 * math.pi, 8)
        bg.append((cx, cy, amp, ph))
    base = g.uniform(0.3, 0.7, 3)
    tex = []
    for ch in range(3):
        lam = g.uniform(24.0, 96.0, 64)
        ang = g.uniform(0.0, 2 * math.pi, 64)
        amp = g.uniform(0.0, 1.0, 64)
        amp *= 0.15 / np.sum(amp)
        ph = g.uniform(0.0, 2 * math.pi, 64)
        tex.append((lam, ang, amp, ph))
    return bg, base, tex


def conferencing_frame(width: int, height: int, seed: int, t: int = 0,
                       motion: SubjectMotion = SubjectMotion(), area_frac: float = 0.3,
                       aspect: float = 1.3, edge_px: float = 1.5):
    """Synthetic video-conferencing frame ``t`` and its region-of-interest mask.

    Returns ``(frame[3, H, W] float32, mask[H, W] bool)``; the mask is the exact
    ellipse of the subject at frame ``t`` (stand-in for a matting network).
    """
    bg_spec, base, tex_spec = _scene_spec(seed)
    # semi-axes: pi * a * b = area_frac * W * H, b = aspect * a (b vertical)
    a = math.sqrt(area_frac * width * height / (math.pi * aspect))
    b = aspect * a
    theta = math.radians(motion.omega * t)
    cx = width / 2.0 + motion.v * t * math.cos(motion.direction)
    cy = height / 2.0 + motion.v * t * math.sin(motion.direction)
    xs = np.arange(width, dtype=np.float64) + 0.5
    ys = np.arange(height, dtype=np.float64) + 0.5
    X, Y = np.meshgrid(xs - cx, ys - cy)
    ct, st = math.cos(theta), math.sin(theta)
    # object coordinates: rotate by -theta
    ox = ct * X + st * Y
    oy = -st * X + ct * Y
    rho = np.sqrt((ox / a) ** 2 + (oy / b) ** 2)
    # signed distance approximation (in px) to the ellipse boundary
    dist = (1.0 - rho) * min(a, b)
    s = np.clip(dist / edge_px * 0.5 + 0.5, 0.0, 1.0)
    alpha = s * s * (3.0 - 2.0 * s)
    frame = np.empty((3, height, width), dtype=np.float64)
    for ch in range(3):
        cxs, cys, amp, ph = bg_spec[ch]
        bgc = 0.5 + 0.25 * _plane_wave_sum(width, height, 2 * math.pi * cxs / width,
                                           2 * math.pi * cys / height, ph, amp) / np.sum(amp)
        lam, ang, tamp, tph = tex_spec[ch]
        # plane wave in object coords k.(R(-theta)(p - c)) = (R(theta) k).p - (R(theta) k).c
        kx0 = 2 * math.pi / lam * np.cos(ang)
        ky0 = 2 * math.pi / lam * np.sin(ang)
        kx = ct * kx0 - st * ky0
        ky = st * kx0 + ct * ky0
        phase = tph - (kx * cx + ky * cy)
        fg = base[ch] + _plane_wave_sum(width, height, kx, ky, phase, tamp)
        frame[ch] = alpha * fg + (1.0 - alpha) * bgc
    mask = rho <= 1.0
    return frame.astype(np.float32), mask


def conferencing_gaussians(frame: np.ndarray, mask: np.ndarray, n: int, seed: int,
                           roi_frac: float = 0.7) -> np.ndarray:
    """Seeded Gaussian set shaped like an ROI-initialised fit of a conferencing
    frame: ``roi_frac`` of the means uniform inside the mask, the rest outside;
    isotropic-ish footprints sized so each Gaussian covers its share of its
    region (variance area / (4 pi), the variance of a disk of that area);
    colour sampled from the frame at the mean; weight 1.  A synthetic stand-in
    for timing and parity work (the initialiser itself is not here)."""
    g = rng(seed)
    _, h, w = frame.shape
    n_roi = int(round(roi_frac * n))
    out = np.empty((9, n), dtype=np.float64)
    ys, xs = np.nonzero(mask)
    yb, xb = np.nonzero(~mask)
    for sl, (py, px) in ((slice(0, n_roi), (ys, xs)), (slice(n_roi, n), (yb, xb))):
        k = sl.stop - sl.start
        if k <= 0:
            continue
        if len(px) == 0:
            py, px = np.nonzero(np.ones_like(mask))
        pick = g.integers(0, len(px), k)
        out[0, sl] = px[pick] + g.uniform(0.0, 1.0, k)
        out[1, sl] = py[pick] + g.uniform(0.0, 1.0, k)
        s = math.sqrt(len(px) / k / (4.0 * math.pi))
        out[2, sl] = s * g.uniform(0.8, 1.25, k)
        out[4, sl] = s * g.uniform(0.8, 1.25, k)
        out[3, sl] = g.normal(0.0, 0.2 * s, k)
    xi = np.clip(out[0].astype(np.int64), 0, w - 1)
    yi = np.clip(out[1].astype(np.int64), 0, h - 1)
    out[5:8] = frame[:, yi, xi]
    out[8] = 1.0
    return out.astype(np.float32)


def block_image(bx: int, by: int, b: int, seed: int = 0):
    """``bx`` x ``by`` blocks of ``b`` x ``b`` constant colours (distinct colours
    from a 4-level lattice per channel, pairwise distance >= 0.3); returns
    ``(image[3, by b, bx b] float32, colours[bx by, 3])``."""
    g = rng(seed)
    levels = (0.1, 0.4, 0.7, 1.0)
    lattice = np.array([(r, gg, bb) for r in levels for gg in levels for bb in levels])
    if bx * by > len(lattice):
        raise ValueError("at most 64 blocks")
    cols = lattice[g.permutation(len(lattice))[:bx * by]]
    img = np.zeros((3, by * b, bx * b), np.float32)
    for j in range(by):
        for i in range(bx):
            img[:, j * b:(j + 1) * b, i * b:(i + 1) * b] = cols[j * bx + i][:, None, None]
    return img, cols


def background_positions(mask: np.ndarray, n: int, seed: int) -> np.ndarray:
    """``[2, n]`` float32 positions uniform over the pixels outside ``mask``
    (a uniformly chosen background pixel plus a uniform offset inside it): the
    random draws of an initialiser's background Gaussians, passed in as input."""
    g = rng(seed)
    ys, xs = np.nonzero(~np.asarray(mask, bool))
    if len(xs) == 0:
        ys, xs = np.nonzero(np.ones_like(mask, bool))
    pick = g.integers(0, len(xs), n)
    out = np.empty((2, n), np.float64)
    out[0] = xs[pick] + g.uniform(0.0, 1.0, n)
    out[1] = ys[pick] + g.uniform(0.0, 1.0, n)
    return out.astype(np.float32)


def conferencing_sequence(width: int, height: int, seed: int, frames: int,
                          motion: SubjectMotion | None = None):
    """Yields ``(frame, mask)`` for ``frames`` frames of one rigidly moving subject."""
    if motion is None:
        motion = random_motion(seed + 7919)
    for t in range(frames):
        yield conferencing_frame(width, height, seed, t, motion)


def clip_table(count: int, seed: int, resolutions=((640, 360), (1280, 720), (1920, 1080)),
               n_range=(2000, 50000)):
    """Batched-encode clip table: list of dicts with ``width, height, n, seed``.

    Resolutions uniform over ``resolutions``; Gaussian counts log-uniform over
    ``n_range`` (inclusive bounds, rounded to an integer).
    """
    g = rng(seed)
    out = []
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    for i in range(count):
        w, h = resolutions[int(g.integers(0, len(resolutions)))]
        n = int(round(math.exp(g.uniform(lo, hi))))
        out.append({"width": w, "height": h, "n": n, "seed": seed * 1000 + i})
    return out
