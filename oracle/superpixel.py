"""Oracle for the region-of-interest superpixel initialiser (Sec. 3.2 A) --
TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper segments the region of interest into N superpixels with a K-means
superpixel algorithm and initialises one Gaussian per segment: mean = segment
centre, Cholesky factor from the segment covariance, colour = mean segment
colour.  It leaves the clustering details, the covariance scale and the
Gaussians outside the region to the reader; the readings implemented here:

* seeds on a square grid of step S = max(1, sqrt(A_roi / K)) (A_roi = mask
  pixels; at most one superpixel per pixel),
  at ((i + 1/2) S, (j + 1/2) S), kept where the seed's pixel is in the mask;
  the number of region Gaussians is the number of seeds M (at most n);
* I = 10 K-means iterations in (r, g, b, x, y): a mask pixel p (centre at
  (x + 1/2, y + 1/2)) joins the centre minimising
      D = |col_p - col_c|^2 + (m / S)^2 |p - c|^2,  m = 0.2,
  among centres within S of p on both axes (ties: lowest index); a centre moves
  to the mean colour and position of its pixels, then is clamped to within S
  of its seed on each axis (so the candidates of p are exactly the seeds whose
  grid cells lie within two cells of p's); a centre without pixels stays;
* each final segment gives a Gaussian with mean = centroid, Sigma =
  kappa (covariance of the pixel centres + I/12), kappa = 4 (I/12 completes
  the second moment of the segment's area: b^2/12 I for a b x b block; kappa
  widens it so that the accumulated sum of Eq. 2 over a tiling of segments is
  flat -- on a square grid of step S with sigma = S/sqrt(3) the ripple is
  about 2 exp(-2 pi^2 kappa / 12) ~ 0.3 %), L = chol(Sigma), colour = mean
  colour, weight w = A / (2 pi sqrt(det Sigma)) so that the Gaussian's
  integral equals the segment area A (the blend keeps the mean level); a
  segment that lost all pixels keeps its seed with Sigma = kappa S^2/12 I, the
  frame colour at the seed and w = 1;
* the remaining n - M Gaussians sit at caller-supplied positions bg_xy
  (random numbers are inputs), isotropic with variance kappa a / (2 pi),
  a = (background pixels) / (n - M), weight 1 / kappa (integral a), colour =
  frame at the mean.

Arithmetic (a reading: the paper fixes no precision).  The assignment's
distances and comparisons are single precision (numpy float32, each
operation rounded once; the centres are kept as float32), the precision the
GPU kernel decides in.  Every sum over a segment is exact: pixel-centre
coordinates enter as the integers 2 x + 1 - 2 floor(seed) (twice the offset
from the seed's pixel), colours as rint(c 2^20) (colours clamped to
[-32, 32]), so counts, first and second moments are integers whose sums do
not depend on their order; means and covariances follow from them by a fixed
sequence of double-precision operations, rounded once to float32 at the end.
"""

from __future__ import annotations

import math

import numpy as np

COMPACTNESS = 0.2
ITERATIONS = 10
KAPPA = 4.0  # covariance scale: keeps the additive blend of a tiling flat
COLOUR_SCALE = float(1 << 20)
COLOUR_LIMIT = 32.0


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


def assign(frame, mask, centers_col, centers_xy, seed_cells, S, m=COMPACTNESS):
    """Label map (int64 [H, W], -1 outside the mask) for the given float32
    centres: a mask pixel joins the candidate minimising, in float32,
    D = ((r - r_c)^2 + (g - g_c)^2) + (b - b_c)^2 + lam ((dx^2 + dy^2)),
    lam = float32((m / S)^2), among centres with |dx|, |dy| <= float32(S);
    candidates are visited in ascending index and only a strictly smaller D
    replaces the best."""
    _, h, w = frame.shape
    label = np.full((h, w), -1, np.int64)
    ys, xs = np.nonzero(mask)          # the mask pixels, raster order
    if len(xs) == 0 or len(centers_xy) == 0:
        return label
    f32 = np.float32
    col = frame[:, ys, xs].astype(f32)
    PX = (xs.astype(np.float64) + 0.5).astype(f32)
    PY = (ys.astype(np.float64) + 0.5).astype(f32)
    S32 = f32(S)
    lam = f32((m / S) * (m / S))
    ccol = np.asarray(centers_col, f32)
    cxy = np.asarray(centers_xy, f32)
    best = np.full(len(xs), np.inf, f32)
    lab = np.full(len(xs), -1, np.int64)
    gx = int(math.ceil(w / S))
    gy = int(math.ceil(h / S))
    cell_of = np.full((gy, gx), -1, np.int64)
    for idx, (i, j) in enumerate(seed_cells):
        cell_of[j, i] = idx
    pcx = np.floor(PX.astype(np.float64) / S).astype(np.int64)
    pcy = np.floor(PY.astype(np.float64) / S).astype(np.int64)
    cand_lists = []
    for dj in range(-2, 3):
        for di in range(-2, 3):
            cx, cy = pcx + di, pcy + dj
            ok = (cx >= 0) & (cx < gx) & (cy >= 0) & (cy < gy)
            idx = np.where(ok, cell_of[np.clip(cy, 0, gy - 1), np.clip(cx, 0, gx - 1)], -1)
            cand_lists.append(idx)
    cand = np.stack(cand_lists, 0)  # [25, P]
    order = np.argsort(np.where(cand < 0, np.iinfo(np.int64).max, cand), axis=0, kind="stable")
    cand = np.take_along_axis(cand, order, 0)
    for k in range(cand.shape[0]):
        idx = cand[k]
        valid = idx >= 0
        if not valid.any():
            break
        ii = np.where(valid, idx, 0)
        dx = PX - cxy[ii, 0]
        dy = PY - cxy[ii, 1]
        within = valid & (np.abs(dx) <= S32) & (np.abs(dy) <= S32)
        dr, dg, db = col[0] - ccol[ii, 0], col[1] - ccol[ii, 1], col[2] - ccol[ii, 2]
        dc = (dr * dr + dg * dg) + db * db
        d = dc + lam * (dx * dx + dy * dy)
        take = within & (d < best)
        best = np.where(take, d, best)
        lab = np.where(take, idx, lab)
    label[ys, xs] = lab
    return label


def segment_sums(frame, label, seeds_xy):
    """Exact integer sums per segment: count, sum of u = 2 x + 1 - 2 floor(qx),
    of v (the same in y), of u^2, u v, v^2 and of rint(c 2^20) per channel
    (object arrays of Python ints, [k])."""
    _, h, w = frame.shape
    k = len(seeds_xy)
    sums = {key: [0] * k for key in ("n", "u", "v", "uu", "uv", "vv", "r", "g", "b")}
    ys, xs = np.nonzero(label >= 0)
    if len(xs) == 0 or k == 0:
        return sums
    lab = label[ys, xs]
    fx = np.floor(np.asarray(seeds_xy)[:, 0]).astype(np.int64)
    fy = np.floor(np.asarray(seeds_xy)[:, 1]).astype(np.int64)
    u = 2 * xs.astype(np.int64) + 1 - 2 * fx[lab]
    v = 2 * ys.astype(np.int64) + 1 - 2 * fy[lab]
    q = [np.rint(np.clip(frame[ch, ys, xs].astype(np.float64), -COLOUR_LIMIT, COLOUR_LIMIT)
                 * COLOUR_SCALE).astype(np.int64) for ch in range(3)]
    for key, vals in (("n", np.ones_like(u)), ("u", u), ("v", v), ("uu", u * u), ("uv", u * v),
                      ("vv", v * v), ("r", q[0]), ("g", q[1]), ("b", q[2])):
        acc = np.zeros(k, np.int64)
        np.add.at(acc, lab, vals)      # int64: exact, order-free
        sums[key] = [int(a) for a in acc]
    return sums


def update(frame, label, centers_col, centers_xy, seeds_xy, S):
    """New float32 centres: the segment's mean position (u / (2 n) + floor(q)
    in double) clamped to within S of the seed, and mean colour (sum /
    (n 2^20) in double); empty segments keep their centre."""
    sm = segment_sums(frame, label, seeds_xy)
    new_col = np.asarray(centers_col, np.float32).copy()
    new_xy = np.asarray(centers_xy, np.float32).copy()
    for c in range(len(seeds_xy)):
        n = sm["n"][c]
        if n == 0:
            continue
        qx, qy = float(seeds_xy[c][0]), float(seeds_xy[c][1])
        mx = float(sm["u"][c]) / float(2 * n) + math.floor(qx)
        my = float(sm["v"][c]) / float(2 * n) + math.floor(qy)
        new_xy[c, 0] = np.float32(min(max(mx, qx - S), qx + S))
        new_xy[c, 1] = np.float32(min(max(my, qy - S), qy + S))
        for ch, key in enumerate(("r", "g", "b")):
            new_col[c, ch] = np.float32(float(sm[key][c]) / (float(n) * COLOUR_SCALE))
    return new_col, new_xy


def segment(frame, mask, k_target, iterations=ITERATIONS, m=COMPACTNESS, max_seeds=None):
    """K-means superpixels of the mask: (S, seeds [M,2], labels [H,W], centres)."""
    frame = np.asarray(frame, np.float32)
    mask = np.asarray(mask, bool)
    S, sxy, cells = seeds(mask, k_target, max_seeds)
    _, h, w = frame.shape
    xi = np.clip(np.floor(sxy[:, 0]).astype(np.int64), 0, w - 1)
    yi = np.clip(np.floor(sxy[:, 1]).astype(np.int64), 0, h - 1)
    ccol = frame[:, yi, xi].T.astype(np.float32)
    cxy = sxy.astype(np.float32)
    label = np.full((h, w), -1, np.int64)
    for it in range(iterations):
        label = assign(frame, mask, ccol, cxy, cells, S, m)
        if it + 1 < iterations:
            ccol, cxy = update(frame, label, ccol, cxy, sxy, S)
    return S, sxy, label, (ccol, cxy)


def gaussians_from_segments(frame, label, sxy, S):
    """[9, M] float64 Gaussians from the final segments (see module doc), from
    the exact integer sums: mean = u / (2 n) + floor(q); covariance of the
    pixel centres (uu / n - (u / n)^2) / 4 etc. in double; Sigma = KAPPA
    (covariance + I/12); L = chol(Sigma); colour = sum / (n 2^20); weight =
    n / (2 pi l1 l3)."""
    _, h, w = frame.shape
    k = len(sxy)
    out = np.zeros((9, k), np.float64)
    sm = segment_sums(frame, label, sxy)
    two_pi = 2.0 * math.pi
    for i in range(k):
        n = sm["n"][i]
        if n == 0:
            xi = min(max(int(math.floor(sxy[i, 0])), 0), w - 1)
            yi = min(max(int(math.floor(sxy[i, 1])), 0), h - 1)
            s = 2.0 * (S / math.sqrt(12.0))
            out[:, i] = [sxy[i, 0], sxy[i, 1], s, 0.0, s, frame[0, yi, xi], frame[1, yi, xi],
                         frame[2, yi, xi], 1.0]
            continue
        fn = float(n)
        au, av = float(sm["u"][i]) / fn, float(sm["v"][i]) / fn
        cxx = (float(sm["uu"][i]) / fn - au * au) / 4.0
        cxy = (float(sm["uv"][i]) / fn - au * av) / 4.0
        cyy = (float(sm["vv"][i]) / fn - av * av) / 4.0
        vxx = cxx + 1.0 / 12.0
        vyy = cyy + 1.0 / 12.0
        l1 = math.sqrt(vxx)
        l2 = cxy / l1
        l3 = math.sqrt(vyy - l2 * l2)
        # Sigma = KAPPA (cov + I/12): the factor sqrt(KAPPA) = 2 is exact
        l1, l2, l3 = 2.0 * l1, 2.0 * l2, 2.0 * l3
        out[0, i] = float(sm["u"][i]) / float(2 * n) + math.floor(sxy[i, 0])
        out[1, i] = float(sm["v"][i]) / float(2 * n) + math.floor(sxy[i, 1])
        out[2, i], out[3, i], out[4, i] = l1, l2, l3
        for ch, key in enumerate(("r", "g", "b")):
            out[5 + ch, i] = float(sm[key][i]) / (fn * COLOUR_SCALE)
        out[8, i] = fn / (two_pi * l1 * l3)
    return out


def background_gaussians(frame, mask, bg_xy, count):
    """[9, count] isotropic Gaussians at bg_xy[:count] (variance a / (2 pi))."""
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
    out[5:8] = frame[:, yi, xi]
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
    return np.concatenate([roi, bg], axis=1), {"S": S, "seeds": sxy, "label": label, "M": M}
