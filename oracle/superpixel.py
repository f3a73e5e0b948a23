"""Oracle for the region-of-interest superpixel initialiser (Sec. 3.2 A) --
TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper segments the region of interest into N superpixels with a K-means
superpixel algorithm and initialises one Gaussian per segment: mean = segment
centre, Cholesky factor from the segment covariance, colour = mean segment
colour.  It leaves the clustering details, the covariance scale and the
Gaussians outside the region to the reader; the readings implemented here:

* seeds on a square grid of step S = sqrt(A_roi / K) (A_roi = mask pixels),
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

All arithmetic is double precision; sums run over pixels in raster order.
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
    S = math.sqrt(area / k_target)
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
    """Label map (int64 [H, W], -1 outside the mask) for the given centres."""
    _, h, w = frame.shape
    label = np.full((h, w), -1, np.int64)
    ys, xs = np.nonzero(mask)          # the mask pixels, raster order
    if len(xs) == 0 or len(centers_xy) == 0:
        return label
    col = frame[:, ys, xs].astype(np.float64)
    PX = xs.astype(np.float64) + 0.5
    PY = ys.astype(np.float64) + 0.5
    best = np.full(len(xs), np.inf)
    lab = np.full(len(xs), -1, np.int64)
    # seed index by grid cell
    gx = int(math.ceil(w / S))
    gy = int(math.ceil(h / S))
    cell_of = np.full((gy, gx), -1, np.int64)
    for idx, (i, j) in enumerate(seed_cells):
        cell_of[j, i] = idx
    pcx = np.floor(PX / S).astype(np.int64)
    pcy = np.floor(PY / S).astype(np.int64)
    lam = (m / S) * (m / S)
    # candidates in ascending centre index: gather the 25 cells, sort by index
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
        dx = PX - centers_xy[ii, 0]
        dy = PY - centers_xy[ii, 1]
        within = valid & (np.abs(dx) <= S) & (np.abs(dy) <= S)
        dc = ((col[0] - centers_col[ii, 0]) ** 2 + (col[1] - centers_col[ii, 1]) ** 2) \
            + (col[2] - centers_col[ii, 2]) ** 2
        d = dc + lam * (dx * dx + dy * dy)
        take = within & (d < best)
        best = np.where(take, d, best)
        lab = np.where(take, idx, lab)
    label[ys, xs] = lab
    return label


def update(frame, label, centers_col, centers_xy, seeds_xy, S):
    """New centres: mean colour and position of each segment (raster-order
    double sums), clamped to within S of the seed; empty segments stay."""
    _, h, w = frame.shape
    k = len(centers_xy)
    lab = label.reshape(-1)
    sel = lab >= 0
    px = (np.arange(w, dtype=np.float64) + 0.5)[None, :].repeat(h, 0).reshape(-1)
    py = (np.arange(h, dtype=np.float64) + 0.5)[:, None].repeat(w, 1).reshape(-1)
    cnt = np.bincount(lab[sel], minlength=k).astype(np.float64)
    new_xy = centers_xy.copy()
    new_col = centers_col.copy()
    nz = cnt > 0
    for d, vals in enumerate((px, py)):
        s = np.bincount(lab[sel], weights=vals[sel], minlength=k)
        new_xy[nz, d] = s[nz] / cnt[nz]
    for ch in range(3):
        v = frame[ch].astype(np.float64).reshape(-1)
        s = np.bincount(lab[sel], weights=v[sel], minlength=k)
        new_col[nz, ch] = s[nz] / cnt[nz]
    new_xy = np.minimum(np.maximum(new_xy, seeds_xy - S), seeds_xy + S)
    return new_col, new_xy


def segment(frame, mask, k_target, iterations=ITERATIONS, m=COMPACTNESS, max_seeds=None):
    """K-means superpixels of the mask: (S, seeds [M,2], labels [H,W], centres)."""
    frame = np.asarray(frame, np.float32)
    mask = np.asarray(mask, bool)
    S, sxy, cells = seeds(mask, k_target, max_seeds)
    _, h, w = frame.shape
    xi = np.clip(np.floor(sxy[:, 0]).astype(np.int64), 0, w - 1)
    yi = np.clip(np.floor(sxy[:, 1]).astype(np.int64), 0, h - 1)
    ccol = frame[:, yi, xi].T.astype(np.float64)
    cxy = sxy.copy()
    label = np.full((h, w), -1, np.int64)
    for _ in range(iterations):
        label = assign(frame, mask, ccol, cxy, cells, S, m)
        ccol, cxy = update(frame, label, ccol, cxy, sxy, S)
    return S, sxy, label, (ccol, cxy)


def gaussians_from_segments(frame, label, sxy, S):
    """[9, M] float64 Gaussians from the final segments (see module doc)."""
    _, h, w = frame.shape
    k = len(sxy)
    out = np.zeros((9, k), np.float64)
    lab = label.reshape(-1)
    sel = lab >= 0
    px = (np.arange(w, dtype=np.float64) + 0.5)[None, :].repeat(h, 0).reshape(-1)
    py = (np.arange(h, dtype=np.float64) + 0.5)[:, None].repeat(w, 1).reshape(-1)
    L = lab[sel]
    cnt = np.bincount(L, minlength=k).astype(np.float64)
    sx = np.bincount(L, weights=px[sel], minlength=k)
    sy = np.bincount(L, weights=py[sel], minlength=k)
    for i in range(k):
        if cnt[i] == 0:
            xi = min(max(int(math.floor(sxy[i, 0])), 0), w - 1)
            yi = min(max(int(math.floor(sxy[i, 1])), 0), h - 1)
            s = 2.0 * (S / math.sqrt(12.0))
            out[:, i] = [sxy[i, 0], sxy[i, 1], s, 0.0, s, frame[0, yi, xi], frame[1, yi, xi],
                         frame[2, yi, xi], 1.0]
    nz = np.nonzero(cnt)[0]
    mx = sx[nz] / cnt[nz]
    my = sy[nz] / cnt[nz]
    # centred second moments (two-pass), raster order
    dxm = px[sel] - (sx / np.maximum(cnt, 1))[L]
    dym = py[sel] - (sy / np.maximum(cnt, 1))[L]
    sxx = np.bincount(L, weights=dxm * dxm, minlength=k)
    sxy_ = np.bincount(L, weights=dxm * dym, minlength=k)
    syy = np.bincount(L, weights=dym * dym, minlength=k)
    vxx = sxx[nz] / cnt[nz] + 1.0 / 12.0
    vxy = sxy_[nz] / cnt[nz]
    vyy = syy[nz] / cnt[nz] + 1.0 / 12.0
    l1 = np.sqrt(vxx)
    l2 = vxy / l1
    l3 = np.sqrt(vyy - l2 * l2)
    # Sigma = KAPPA (cov + I/12): the factor sqrt(KAPPA) = 2 is exact
    l1, l2, l3 = 2.0 * l1, 2.0 * l2, 2.0 * l3
    out[0, nz] = mx
    out[1, nz] = my
    out[2, nz] = l1
    out[3, nz] = l2
    out[4, nz] = l3
    for ch in range(3):
        v = frame[ch].astype(np.float64).reshape(-1)
        out[5 + ch, nz] = np.bincount(L, weights=v[sel], minlength=k)[nz] / cnt[nz]
    out[8, nz] = cnt[nz] / (2.0 * math.pi * l1 * l3)
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
