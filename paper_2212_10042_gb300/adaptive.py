"""Adaptive calibration: pilot simulations choose each tile's size and number of
simulations.

The paper's Phase II/III calibration (Sec. 10.2) uses large tiles and few
simulations where the Type I Error is low and small tiles with many simulations
where it is high, chosen from pilot simulations, but does not state the rule.
Calibration sets lambda* = min_i lambda_i (Eq. calibrated-threshold-final), so
only the tiles whose lambda_i is at or near the minimum decide the result, and
refining a tile raises its lambda_i: a smaller tile has less Tilt-Bound slack
(alpha'_i moves up towards alpha, Eq. tile-calibration-final), more
simulations make k_i / (K_i + 1) track alpha'_i more closely and give
lambda_i = -inf tiles (k_i = 0) an order statistic.  The rule used here:

1. calibrate the current platten (alpha'_i, lambda_i; lambda* = min);
2. a tile is *critical* when lambda_i is among the lowest `crit_frac` of all
   tiles or within `crit_margin` of lambda*;
3. a critical tile with lambda_i = -inf (k_i = 0: too few simulations for an
   order statistic) doubles its number of simulations while K_i < `K_cap`
   (CRN: the tile then uses sims 0 .. 2 K_i - 1); any other critical tile with
   slack (alpha - alpha'_i) / alpha above `slack_tol` splits into its 2^d
   children (half the half-width on every arm; children that do not meet the
   null set are dropped), unless that would take a half-width below
   `min_halfwidth`; otherwise, while K_i < `K_cap`, its K doubles;
4. repeat until no critical tile changes or `max_iter` rounds have run.

Every decision is a comparison of the calibrator's outputs, so two calibrators
that agree (the GPU path and the oracle) produce the same sequence of plattens.
"""
import dataclasses
from typing import Callable, List, Tuple

import numpy as np

from . import workloads as W


@dataclasses.dataclass
class RefineConfig:
    alpha: float = 0.025
    max_iter: int = 6
    crit_frac: float = 0.05
    crit_margin: float = 0.0
    slack_tol: float = 0.1
    min_halfwidth: float = 1.0 / 512
    K_cap: int = 1 << 16


def split(tiles: W.TileSet, rows, one_arm: bool) -> W.TileSet:
    """The 2^d children of each row's box (centre c + s h/2, half-width h/2 for
    s in {-1, +1}^d) that still meet the null set, with the parent's K."""
    rows = np.asarray(rows, dtype=np.int64)
    d = tiles.d
    if rows.size == 0:
        return W.from_centers(np.zeros((0, d)), np.zeros((0, d)), np.zeros(0, np.uint32), np.zeros(0, np.int32))
    c = tiles.centers[rows]
    h = tiles.halfwidth[rows]
    signs = np.array([[1.0 if (m >> a) & 1 else -1.0 for a in range(d)] for m in range(1 << d)])
    cc = (c[:, None, :] + signs[None, :, :] * (0.5 * h)[:, None, :]).reshape(-1, d)
    hh = np.repeat(0.5 * h, 1 << d, axis=0)
    KK = np.repeat(tiles.K[rows], 1 << d)
    nm = W.null_mask_of_boxes(cc, hh, one_arm=one_arm)
    keep = nm != 0
    return W.from_centers(cc[keep], hh[keep], nm[keep], KK[keep])


def concat(parts: List[W.TileSet], d: int) -> W.TileSet:
    parts = [p for p in parts if p.n_tiles > 0]
    if not parts:
        return W.from_centers(np.zeros((0, d)), np.zeros((0, d)), np.zeros(0, np.uint32), np.zeros(0, np.int32))
    c = np.concatenate([p.centers for p in parts])
    h = np.concatenate([p.halfwidth for p in parts])
    nm = np.concatenate([p.null_mask for p in parts])
    K = np.concatenate([p.K for p in parts])
    return W.from_centers(c, h, nm, K)


def critical(lam_tile: np.ndarray, cfg: RefineConfig) -> np.ndarray:
    """Tiles whose lambda_i can set lambda*: the lowest crit_frac, or within
    crit_margin of the minimum (ties at the cut included)."""
    lam = np.asarray(lam_tile, dtype=np.float64)
    lo = lam.min()
    cut = np.quantile(lam, cfg.crit_frac, method="inverted_cdf")
    if np.isfinite(lo):
        cut = max(cut, lo + cfg.crit_margin)
    return lam <= cut


def refine(tiles: W.TileSet, alpha_prime: np.ndarray, lam_tile: np.ndarray, cfg: RefineConfig,
           one_arm: bool) -> Tuple[W.TileSet, int, int]:
    """One round of the rule: returns the new platten, tiles split, tiles whose K doubled."""
    crit = critical(lam_tile, cfg)
    slack = (cfg.alpha - np.asarray(alpha_prime)) / cfg.alpha
    can_split = np.all(0.5 * tiles.halfwidth >= cfg.min_halfwidth, axis=1)
    no_stat = crit & np.isneginf(np.asarray(lam_tile)) & (tiles.K < cfg.K_cap)
    do_split = crit & ~no_stat & (slack > cfg.slack_tol) & can_split
    do_double = crit & ~do_split & (tiles.K < cfg.K_cap)
    K = tiles.K.copy()
    K[do_double] = np.minimum(2 * K[do_double], cfg.K_cap).astype(np.int32)
    kept = np.flatnonzero(~do_split)
    kept_tiles = W.from_centers(tiles.centers[kept], tiles.halfwidth[kept], tiles.null_mask[kept], K[kept])
    children = split(tiles, np.flatnonzero(do_split), one_arm)
    return concat([kept_tiles, children], tiles.d), int(do_split.sum()), int(do_double.sum())


def run(tiles: W.TileSet, calibrate: Callable, cfg: RefineConfig, one_arm: bool) -> dict:
    """The loop.  `calibrate(tiles) -> (alpha_prime, lambda_tile, lambda_star)` as
    numpy arrays and a float.  Returns the last platten, its calibration, and a
    trace of every round (tiles, sum of K, lambda*, tiles split, K doubled)."""
    trace = []
    for it in range(cfg.max_iter):
        ap, lt, lam = calibrate(tiles)
        new, n_split, n_double = refine(tiles, ap, lt, cfg, one_arm)
        trace.append(dict(iteration=it, tiles=tiles.n_tiles, sum_K=int(tiles.K.astype(np.int64).sum()),
                          lam=float(lam), split=n_split, doubled=n_double))
        if n_split == 0 and n_double == 0:
            return dict(tiles=tiles, alpha_prime=ap, lambda_tile=lt, lam=float(lam), trace=trace, converged=True)
        tiles = new
    ap, lt, lam = calibrate(tiles)
    trace.append(dict(iteration=cfg.max_iter, tiles=tiles.n_tiles, sum_K=int(tiles.K.astype(np.int64).sum()),
                      lam=float(lam), split=0, doubled=0))
    return dict(tiles=tiles, alpha_prime=ap, lambda_tile=lt, lam=float(lam), trace=trace, converged=False)


class GpuCalibrator:
    """calibrate() for `run` on the GPU path (cse_calibrate through the binding)."""

    def __init__(self, design: W.Design, alpha: float, K_cap: int, seed: int = None):
        from . import binding
        self._B = binding
        self.alpha = float(alpha)
        self.ctx = binding.Context(design, seed=seed, K_max=K_cap)

    def __call__(self, tiles: W.TileSet):
        dt = self._B.DeviceTiles(tiles)
        cal = self.ctx.calibrate(dt, self.alpha)
        return (cal["alpha_prime"].cpu().numpy(), cal["lambda_tile"].cpu().numpy(), cal["lam"])
