"""Pins for the oracle's tile binning: the single-precision rectangle rule,
worked by hand from its definition, and the coverage property that makes
tiling exact (every contributing pixel of a Gaussian lies in a listed tile)."""

import numpy as np
import pytest

from gs2d_inputs import random_gaussians


def one32(mx, my, l1, l2, l3, w=0.7):
    return np.array([[mx], [my], [l1], [l2], [l3], [0.5], [0.5], [0.5], [w]], np.float32)


# Hand-worked examples of the rule (half-extents rx = ceil(3 sqrt(Sxx)),
# ry = ceil(3 sqrt(Syy)) of the sigma <= 4.5 ellipse, pixel span
# floor(mu -+ r) clipped to the image, tiles of 16 px):
#  A: mu=(100.3, 50.7), l=(2,0,2): Sxx=Syy=4 -> rx=ry=6;
#     x 94..106 -> tiles 5..6, y 44..56 -> tiles 2..3.
#  B: mu=(3, 250), l=(1,0,1): rx=ry=3; x 0..6 -> tile 0; y 247..253 -> tile 15.
#  C: mu=(128, 128), l=(4,3,2): Sxx=16 -> rx=12, Syy=13 -> 3 sqrt=10.82 -> ry=11;
#     x 116..140 -> tiles 7..8, y 117..139 -> tiles 7..8.
#  D: |w| < 1/255, det <= 1e-8, NaN, entirely left of the image -> culled.
CASES = [
    (one32(100.3, 50.7, 2, 0, 2), (5, 2, 7, 4), 4),
    (one32(3.0, 250.0, 1, 0, 1), (0, 15, 1, 16), 1),
    (one32(128.0, 128.0, 4, 3, 2), (7, 7, 9, 9), 4),
    (one32(50, 50, 2, 0, 2, w=0.001), (0, 0, 0, 0), 0),
    (one32(50, 50, 1e-5, 0, 1e-5), (0, 0, 0, 0), 0),
    (one32(np.nan, 50, 2, 0, 2), (0, 0, 0, 0), 0),
    (one32(-50, 10, 1, 0, 1), (0, 0, 0, 0), 0),
]


@pytest.mark.parametrize("p,rect,count", CASES)
def test_hand_worked_rectangles(oracle, p, rect, count):
    r, c, total = oracle.tile_rects(p, 256, 256)
    assert tuple(r[0]) == rect
    assert c[0] == count and total == count


def test_ragged_image_clips_to_last_partial_tile(oracle):
    # W=100 -> 7 tile columns (the last holds 4 px); a Gaussian right of x=99 is culled
    r, c, _ = oracle.tile_rects(one32(98.0, 5.0, 1, 0, 1), 100, 70)
    assert tuple(r[0]) == (5, 0, 7, 1)
    _, c2, _ = oracle.tile_rects(one32(110.0, 5.0, 1, 0, 1), 100, 70)
    assert c2[0] == 0


def test_sorted_keys_and_ranges_are_consistent(oracle):
    W, H = 100, 70
    p = random_gaussians(150, W, H, seed=31)
    keys, ranges = oracle.sorted_keys(p, W, H)
    assert np.all(np.diff(keys.astype(np.int64)) > 0)  # strictly ascending, unique
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    for t in range(ranges.shape[0]):
        s, e = ranges[t]
        assert np.all(tiles[s:e] == t)
        assert (e - s) == np.count_nonzero(tiles == t)
    rect, count, total = oracle.tile_rects(p, W, H)
    assert total == len(keys) == count.sum()


def test_nonfinite_colour_is_culled(oracle):
    p = one32(50, 50, 2, 0, 2)
    p[6, 0] = np.nan
    _, c, total = oracle.tile_rects(p, 256, 256)
    assert c[0] == 0 and total == 0


@pytest.mark.parametrize("sigma_cut", [4.5, 8.0])
def test_coverage_every_contributing_pair_is_listed(oracle, sigma_cut):
    """Tiling is exact: each pixel where Gaussian n contributes (brute force,
    double precision, including the ambiguity band) lies in a tile of n's list,
    for the default cut-off and a wider one (radius sqrt(2 sigma_cut lambda))."""
    W, H, T = 100, 70, 16
    cfg = oracle.Config(sigma_cut=sigma_cut, alpha_min=1e-6)
    p = random_gaussians(120, W, H, seed=37)
    p[2:5] *= 1.7  # larger footprints, more tile crossings
    keys, _ = oracle.sorted_keys(p, W, H, cfg)
    listed = {}
    for k in keys:
        listed.setdefault(int(k & np.uint64(0xFFFFFFFF)), set()).add(int(k >> np.uint64(32)))
    TX = (W + T - 1) // T
    for i in range(p.shape[1]):
        img, lo, hi = oracle.render(p[:, i:i + 1], W, H, cfg, ambiguity=True)
        touched = np.nonzero(np.abs(img[0]) + np.abs(lo[0]) + np.abs(hi[0]) + np.abs(img[1]))
        tiles = set((touched[0] // T) * TX + touched[1] // T)
        assert tiles <= listed.get(i, set()), f"Gaussian {i} not covered"
