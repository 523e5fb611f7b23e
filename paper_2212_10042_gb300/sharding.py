"""Sharding a platten across ranks (one process per GPU).

Tiles are independent problems (Sec. 6.3 / 7.3): each rank simulates and bounds
its own contiguous range of tiles with no data exchange.  Calibration has one
real exchange step, the minimum over tiles of the per-tile thresholds
(Eq. calibrated-threshold-final), done here as one all-reduce MIN of a single
double.  Ranges are balanced by the number of simulations sum_i K_i.
"""
from __future__ import annotations

import math
from typing import Callable, List, Tuple

import numpy as np


def shard_bounds(K, world: int) -> List[Tuple[int, int]]:
    """Contiguous tile ranges [lo, hi) whose sums of K are as equal as possible."""
    K = np.asarray(K, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    cum = np.concatenate([[0], np.cumsum(K)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(cum, total * r / world, side="left")))
    cuts.append(len(K))
    cuts = np.maximum.accumulate(np.minimum(np.asarray(cuts), len(K)))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def calibrate_sharded(shard_fn: Callable[[int, int], np.ndarray], K, rank: int, world: int,
                      group=None, device="cpu"):
    """Per-tile thresholds of this rank's range and the global minimum.

    shard_fn(lo, hi) returns the per-tile lambda of tiles lo..hi-1 (e.g. through
    cse_calibrate on that range).  Returns (lo, hi, lambda_tile, lambda_star).
    """
    import torch
    import torch.distributed as dist

    lo, hi = shard_bounds(K, world)[rank]
    lam = np.asarray(shard_fn(lo, hi), dtype=np.float64) if hi > lo else np.zeros(0)
    m = torch.tensor([lam.min() if lam.size else math.inf], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(m, op=dist.ReduceOp.MIN, group=group)
    return lo, hi, lam, float(m.item())
