"""Sharding a batch of independent clips over ranks (one process per GPU).

Clips share nothing: every step of the path runs per clip, so a batch splits
into per-rank sub-batches with no exchange during the fit; only the timings
are gathered afterwards.  The split balances an estimate of each clip's
per-iteration work, taken before any fitting: the fused render dominates and
scales with the frame's pixels (each pixel visits the Gaussians listed in its
tile), binning and the per-Gaussian reduction scale with the Gaussian count.
"""

from __future__ import annotations

# per-iteration cost of one Gaussian relative to one pixel (projection,
# binning entries, per-pair records and their reduction, Adam)
GAUSSIAN_WEIGHT = 16.0


def clip_cost(width: int, height: int, n: int) -> float:
    """Estimated per-iteration work of a clip, in pixel units."""
    return float(width) * float(height) + GAUSSIAN_WEIGHT * float(n)


def partition_clips(sizes, world: int) -> list[list[int]]:
    """Indices of ``sizes`` = [(width, height, n), ...] for each of ``world``
    ranks: longest-processing-time first (clips by decreasing cost, each to
    the rank with the least load so far, the lower rank on ties), every clip
    exactly once, each rank's list in ascending clip order.  Deterministic, so
    every rank computes the same split on its own."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = [clip_cost(w, h, n) for (w, h, n) in sizes]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def shard_loads(sizes, parts) -> list[float]:
    """Estimated per-iteration work of each rank's share."""
    return [sum(clip_cost(*sizes[i]) for i in p) for p in parts]
