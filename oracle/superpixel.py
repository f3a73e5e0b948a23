"""Oracle for the region-of-interest superpixel initialiser (Sec. 3.2 A) --
TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper segments the region of interest into N superpixels with a K-means
superpixel algorithm and initialises one Gaussian per segment: mean = segment
centre, Cholesky factor from the segment covariance, colour = mean segment
colour.  It leaves the clustering details, the covariance scale and the
Gaussians outside the region to the reader; the readings written out here:

* seeds on a square grid of step S = max(1, sqrt(A_roi / K)) (A_roi = mask
  pixels; at most one superpixel per pixel),
  at ((i + 1/2) S, (j + 1/2) S), kept where the seed's pixel is in the mask,
  numbered in raster order of the grid; the number of region Gaussians is the
  number of seeds M (at most n);
* I = 10 K-means iterations in (r, g, b, x, y): a mask pixel p (centre at
  (x + 1/2, y + 1/2)) joins the centre minimising
      D = |col_p - col_c|^2 + (m / S)^2 |p - c|^2,  m = 0.2,
  among the centres within S of p on both axes (exact ties: the lowest
  index); a centre then moves to the mean colour and the mean pixel centre of
  its segment, clamped to within S of its seed on each axis; a centre without
  pixels stays where it is;
* each final segment gives a Gaussian with mean = mean pixel centre,
  Sigma = kappa (covariance of the pixel centres + I/12), kappa = 4 (I/12
  completes the second moment of the segment's area: b^2/12 I for a b x b
  block; kappa widens it so that the accumulated sum of Eq. 2 over a tiling
  of segments is flat -- on a square grid of step S with sigma = S/sqrt(3)
  the ripple is about 2 exp(-2 pi^2 kappa / 12) ~ 0.3 %), L = chol(Sigma)
  (Eq. 1), colour = mean colour, weight w = A / (2 pi sqrt(det Sigma)) so
  that the Gaussian's integral equals the segment area A; a segment that lost
  all pixels keeps its seed with Sigma = kappa S^2/12 I, the frame colour at
  the seed and w = 1;
* the remaining n - M Gaussians sit at caller-supplied positions bg_xy
  (random numbers are inputs), isotropic with variance kappa a / (2 pi),
  a = (background pixels) / (n - M), weight 1 / kappa (integral a), colour =
  frame at the mean.

Arithmetic: the plain definition in double precision -- distances, means and
covariances are computed from the pixels of each segment with numpy float64
operations.  The paper fixes no precision; an implementation that decides in
single precision may choose either centre where two distances lie within its
rounding error of each other (``assign`` reports the two best distances so a
check can tell such near-ties apart).

The candidate set: the clamp keeps every centre within S of its seed, so a
centre within S of pixel p (per axis) has its seed within 2 S of p, i.e. in
one of the 5 x 5 grid cells around p's cell.  ``assign`` therefore scans those
cells only; that restriction is exact, not an approximation.
"""

from __future__ import annotations

import math

import numpy as np

COMPACTNESS = 0.2
ITERATIONS = 10
KAPPA = 4.0  # covariance scale: keeps the additive blend of a tiling flat


def seeds(mask: np.ndarray, k_target: int, max_seeds: int | None = None):
    """Grid step S and the seed positions (float64 [M, 2]) with their grid cells
    (raster order of the grid; at most max_seeds)."""
    h, w = mask.shape
    area = int(mask.sum())
    if area == 0 or k_target <= 0:
        return 1.0, np.zeros((0, 2)), np.zeros((0, 2), np.int64)
    # a grid finer than the pixels would put several seeds in one pixel: the
    # step is at least one pixel (at most one superpixel per ROI pixel)
    S = max(1.0, math.sqrt(area / k_target))
    gx = int(math.ceil(w / S))
    gy = int(math.ceil(h / S))
    pts, cells = [], []
    for j in range(gy):
        for i in range(gx):
            x, y = (i + 0.5) * S, (j + 0.5) * S
            xi, yi = int(math.floor(x)), int(math.floor(y))
            if xi < w and yi < h and mask[yi, xi] and (max_seeds is None or len(pts) < max_seeds):
                pts.append((x, y))
                cells.append((i, j))
    return S, np.array(pts, np.float64).reshape(-1, 2), np.array(cells, np.int64).reshape(-1, 2)


def _candidates(xs, ys, seed_cells, S, w, h):
    """[25, P] candidate centre indices of the pixels (x, y) (the seeds of the
    5 x 5 cells around each pixel's cell, -1 where none), ascending per pixel."""
    gx = int(math.ceil(w / S))
    gy = int(math.ceil(h / S))
    cell_of = np.full((gy, gx), -1, np.int64)
    for idx, (i, j) in enumerate(seed_cells):
        cell_of[j, i] = idx
    pcx = np.floor((xs + 0.5) / S).astype(np.int64)
    pcy = np.floor((ys + 0.5) / S).astype(np.int64)
    lists = []
    for dj in range(-2, 3):
        for di in range(-2, 3):
            cx, cy = pcx + di, pcy + dj
            ok = (cx >= 0) & (cx < gx) & (cy >= 0) & (cy < gy)
            lists.append(np.where(ok, cell_of[np.clip(cy, 0, gy - 1), np.clip(cx, 0, gx - 1)], -1))
    cand = np.stack(lists, 0)
    key = np.where(cand < 0, np.iinfo(np.int64).max, cand)
    return np.take_along_axis(cand, np.argsort(key, axis=0, kind="stable"), 0)


def assign(frame, mask, centers_col, centers_xy, seed_cells, S, m=COMPACTNESS, with_gap=False):
    """The assignment step (double precision): label map (int64 [H, W], -1
    outside the mask; a mask pixel with no centre within S also gets -1).
    With ``with_gap`` also returns the smallest and the second smallest
    distance of every pixel ([H, W] float64 each, inf where absent)."""
    _, h, w = frame.shape
    label = np.full((h, w), -1, np.int64)
    d1 = np.full((h, w), np.inf)
    d2 = np.full((h, w), np.inf)
    ys, xs = np.nonzero(mask)          # the mask pixels, raster order
    if len(xs) == 0 or len(centers_xy) == 0:
        return (label, d1, d2) if with_gap else label
    col = np.asarray(frame, np.float64)[:, ys, xs]
    px, py = xs + 0.5, ys + 0.5
    ccol = np.asarray(centers_col, np.float64)
    cxy = np.asarray(centers_xy, np.float64)
    lam = (m / S) ** 2
    best = np.full(len(xs), np.inf)
    second = np.full(len(xs), np.inf)
    lab = np.full(len(xs), -1, np.int64)
    cand = _candidates(xs, ys, seed_cells, S, w, h)
    for k in range(cand.shape[0]):
        idx = cand[k]
        valid = idx >= 0
        if not valid.any():
            break
        ii = np.where(valid, idx, 0)
        dx = px - cxy[ii, 0]
        dy = py - cxy[ii, 1]
        within = valid & (np.abs(dx) <= S) & (np.abs(dy) <= S)
        d = ((col[0] - ccol[ii, 0]) ** 2 + (col[1] - ccol[ii, 1]) ** 2
             + (col[2] - ccol[ii, 2]) ** 2) + lam * (dx * dx + dy * dy)
        d = np.where(within, d, np.inf)
        take = d < best                # candidates ascend: ties keep the lower index
        second = np.where(take, best, np.minimum(second, d))
        best = np.where(take, d, best)
        lab = np.where(take, idx, lab)
    label[ys, xs] = lab
    d1[ys, xs] = best
    d2[ys, xs] = second
    return (label, d1, d2) if with_gap else label


def segment_means(frame, label, k):
    """Per segment 0..k-1: pixel count, mean pixel centre (x, y) and mean
    colour (r, g, b), plain float64 means over the segment's pixels
    (count 0: NaN means)."""
    ys, xs = np.nonzero(label >= 0)
    lab = label[ys, xs]
    cnt = np.bincount(lab, minlength=k).astype(np.float64)[:k]
    with np.errstate(invalid="ignore", divide="ignore"):
        mx = np.bincount(lab, weights=xs + 0.5, minlength=k)[:k] / cnt
        my = np.bincount(lab, weights=ys + 0.5, minlength=k)[:k] / cnt
        mc = np.stack([np.bincount(lab, weights=np.asarray(frame[ch], np.float64)[ys, xs],
                                   minlength=k)[:k] / cnt for ch in range(3)], 1)
    return cnt, np.stack([mx, my], 1), mc


def update(frame, label, centers_col, centers_xy, seeds_xy, S):
    """The update step: every centre with pixels moves to its segment's mean
    colour and mean pixel centre, the position clamped to within S of its
    seed on each axis; empty segments keep their centre.  Float64 out."""
    k = len(seeds_xy)
    cnt, mxy, mc = segment_means(frame, label, k)
    new_col = np.array(centers_col, np.float64, copy=True)
    new_xy = np.array(centers_xy, np.float64, copy=True)
    has = cnt > 0
    q = np.asarray(seeds_xy, np.float64)
    new_xy[has] = np.clip(mxy[has], q[has] - S, q[has] + S)
    new_col[has] = mc[has]
    return new_col, new_xy


def initial_centres(frame, sxy):
    """Centres before the first assignment: at the seeds, with the frame's
    colour at the seed's pixel."""
    _, h, w = frame.shape
    xi = np.clip(np.floor(sxy[:, 0]).astype(np.int64), 0, w - 1)
    yi = np.clip(np.floor(sxy[:, 1]).astype(np.int64), 0, h - 1)
    return np.asarray(frame, np.float64)[:, yi, xi].T.copy(), np.array(sxy, np.float64)


def segment(frame, mask, k_target, iterations=ITERATIONS, m=COMPACTNESS, max_seeds=None):
    """K-means superpixels of the mask: (S, seeds [M,2], labels [H,W], centres
    (colour [M,3], position [M,2]) used by the last assignment)."""
    mask = np.asarray(mask, bool)
    S, sxy, cells = seeds(mask, k_target, max_seeds)
    _, h, w = frame.shape
    ccol, cxy = initial_centres(frame, sxy)
    label = np.full((h, w), -1, np.int64)
    for it in range(iterations):
        label = assign(frame, mask, ccol, cxy, cells, S, m)
        if it + 1 < iterations:
            ccol, cxy = update(frame, label, ccol, cxy, sxy, S)
    return S, sxy, label, (ccol, cxy)


def gaussians_from_segments(frame, label, sxy, S):
    """[9, M] float64 Gaussians from the final segments (see module doc): mean
    of the pixel centres, population covariance of the pixel centres, Sigma =
    KAPPA (covariance + I/12), L = chol(Sigma) (Eq. 1), mean colour, weight
    n / (2 pi sqrt(det Sigma)) = n / (2 pi l1 l3)."""
    frame = np.asarray(frame, np.float64)
    _, h, w = frame.shape
    k = len(sxy)
    out = np.zeros((9, k), np.float64)
    ys, xs = np.nonzero(label >= 0)
    lab = label[ys, xs]
    order = np.argsort(lab, kind="stable")
    lab, xs, ys = lab[order], xs[order], ys[order]
    starts = np.searchsorted(lab, np.arange(k + 1))
    for i in range(k):
        a, b = starts[i], starts[i + 1]
        if a == b:
            xi = min(max(int(math.floor(sxy[i, 0])), 0), w - 1)
            yi = min(max(int(math.floor(sxy[i, 1])), 0), h - 1)
            s = math.sqrt(KAPPA * S * S / 12.0)
            out[:, i] = [sxy[i, 0], sxy[i, 1], s, 0.0, s, frame[0, yi, xi], frame[1, yi, xi],
                         frame[2, yi, xi], 1.0]
            continue
        px, py = xs[a:b] + 0.5, ys[a:b] + 0.5
        n = float(b - a)
        mx, my = px.mean(), py.mean()
        cxx = np.mean((px - mx) ** 2)
        cxy = np.mean((px - mx) * (py - my))
        cyy = np.mean((py - my) ** 2)
        sxx = KAPPA * (cxx + 1.0 / 12.0)
        sxy_ = KAPPA * cxy
        syy = KAPPA * (cyy + 1.0 / 12.0)
        l1 = math.sqrt(sxx)
        l2 = sxy_ / l1
        l3 = math.sqrt(syy - l2 * l2)
        out[0, i], out[1, i] = mx, my
        out[2, i], out[3, i], out[4, i] = l1, l2, l3
        for ch in range(3):
            out[5 + ch, i] = frame[ch, ys[a:b], xs[a:b]].mean()
        out[8, i] = n / (2.0 * math.pi * l1 * l3)
    return out


def background_gaussians(frame, mask, bg_xy, count):
    """[9, count] isotropic Gaussians at bg_xy[:count] (variance KAPPA a / (2 pi))."""
    _, h, w = frame.shape
    out = np.zeros((9, count), np.float64)
    if count <= 0:
        return out
    a = float((~np.asarray(mask, bool)).sum()) / count
    s = math.sqrt(KAPPA * max(a, 1.0) / (2.0 * math.pi))
    xy = np.asarray(bg_xy, np.float64)[:count]
    xi = np.clip(np.floor(xy[:, 0]).astype(np.int64), 0, w - 1)
    yi = np.clip(np.floor(xy[:, 1]).astype(np.int64), 0, h - 1)
    out[0] = xy[:, 0]
    out[1] = xy[:, 1]
    out[2] = s
    out[4] = s
    out[5:8] = np.asarray(frame, np.float64)[:, yi, xi]
    out[8] = 1.0 / KAPPA
    return out


def roi_init(frame, mask, n, roi_frac, bg_xy, iterations=ITERATIONS, m=COMPACTNESS):
    """The full initialiser: [9, n] float64 (region Gaussians first), plus the
    segmentation for inspection."""
    frame = np.asarray(frame, np.float32)
    mask = np.asarray(mask, bool)
    k_target = int(round(roi_frac * n))
    S, sxy, label, centres = segment(frame, mask, k_target, iterations, m, max_seeds=n)
    M = len(sxy)
    roi = gaussians_from_segments(frame, label, sxy, S)
    bg = background_gaussians(frame, mask, bg_xy, n - M)
    return np.concatenate([roi, bg], axis=1), {"S": S, "seeds": sxy, "label": label, "M": M,
                                               "centres": centres}
