"""Position sharding across ranks (one GPU per rank, no collective on the data path).

Cutouts are independent (Eqs. 21-22 per position), so a batch splits into
contiguous, nearly equal position ranges, balanced by pixel count; each rank
evaluates its range into its own packed output and the caller reassembles the
ranks' outputs in rank order.
"""
from __future__ import annotations

import numpy as np


def shard_ranges(npix, world: int):
    """[start, stop) position ranges per rank, contiguous, balanced by N^2."""
    npix = np.asarray(npix, np.int64)
    if world < 1:
        raise ValueError("world size must be >= 1")
    w = npix * npix
    cum = np.concatenate([[0], np.cumsum(w)])
    total = cum[-1]
    bounds = [0]
    for r in range(1, world):
        bounds.append(int(np.searchsorted(cum, total * r / world, side="left")))
    bounds.append(len(npix))
    bounds = np.maximum.accumulate(np.minimum(bounds, len(npix)))
    return [(int(bounds[r]), int(bounds[r + 1])) for r in range(world)]


def shard(lm, npix, rank: int, world: int):
    """This rank's positions and sizes, and the packed offset of its first pixel."""
    lm = np.asarray(lm, np.float64).reshape(-1, 2)
    npix = np.asarray(npix, np.int32)
    a, b = shard_ranges(npix, world)[rank]
    first = int((npix[:a].astype(np.int64) ** 2).sum())
    return lm[a:b], npix[a:b], first
