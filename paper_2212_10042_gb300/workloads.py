"""Seeded synthetic designs and tile sets (plattens) for the CSE hot path.

Input construction only: grids, box half-widths, null-configuration masks and
simulation counts.  Nothing here evaluates the method (no uniforms, no
statistics, no bounds).  Both the CUDA path and the CPU oracle take their inputs
from here.

Tile convention (Def. tile/platten): a tile is the box
[c - h, c + h] (per arm) around its simulation point c (the box centre,
Sec. 6.2 "choose theta_0 close to H, e.g. the center").  Hypothesis H_j is
"theta_j <= theta_0" (treatment j no better than control; for the one-arm
design "theta <= 0").  A tile's null mask has bit j-1 set when the OPEN box
meets H_j; tiles meeting no hypothesis are not part of the platten.

Tile sets are stored in an axis-indexed form: per arm, the sorted distinct
centre coordinates ("axis"), and per tile an index into that axis.  Every
platten built from a lattice (all workloads below) has few distinct
coordinates per arm.
"""
from __future__ import annotations

import dataclasses
import heapq
from typing import List

import numpy as np


@dataclasses.dataclass(frozen=True)
class Design:
    name: str
    stat: str            # "one_arm_z" | "two_arm_pooled_z" | "bayes4" | "berry4"
    d: int               # arms
    looks: tuple         # cumulative patients per arm at each analysis
    seed: int = 0
    p0: float = 0.5      # one-arm null proportion
    drop: float = 0.1    # bayes4 interim drop threshold
    arm_null: tuple = (0.0, 0.0, 0.0, 0.0)   # berry4: logit of each arm's null response rate

    @property
    def n_max(self) -> int:
        return self.looks[-1]


@dataclasses.dataclass
class TileSet:
    d: int
    axis: List[np.ndarray]       # per arm: sorted distinct centre coordinates (float64)
    idx: np.ndarray              # [n_tiles, d] int32
    halfwidth: np.ndarray        # [n_tiles, d] float64
    null_mask: np.ndarray        # [n_tiles] uint32
    K: np.ndarray                # [n_tiles] int32

    @property
    def n_tiles(self) -> int:
        return int(self.K.shape[0])

    @property
    def centers(self) -> np.ndarray:
        return np.stack([self.axis[a][self.idx[:, a]] for a in range(self.d)], axis=1)

    @property
    def K_max(self) -> int:
        return int(self.K.max())

    def subset(self, rows) -> "TileSet":
        rows = np.asarray(rows)
        return TileSet(self.d, self.axis, np.ascontiguousarray(self.idx[rows]),
                       np.ascontiguousarray(self.halfwidth[rows]),
                       np.ascontiguousarray(self.null_mask[rows]),
                       np.ascontiguousarray(self.K[rows]))

    def with_K(self, K) -> "TileSet":
        Ka = np.broadcast_to(np.asarray(K, dtype=np.int32), self.K.shape).copy()
        return TileSet(self.d, self.axis, self.idx, self.halfwidth, self.null_mask, Ka)


def from_centers(centers, halfwidth, null_mask, K) -> TileSet:
    """Axis-indexed tile set from explicit centres [n, d]."""
    centers = np.asarray(centers, dtype=np.float64)
    n, d = centers.shape
    axis, idx = [], np.zeros((n, d), dtype=np.int32)
    for a in range(d):
        u, inv = np.unique(centers[:, a], return_inverse=True)
        axis.append(u.astype(np.float64))
        idx[:, a] = inv.astype(np.int32)
    hw = np.broadcast_to(np.asarray(halfwidth, dtype=np.float64), (n, d)).copy()
    nm = np.broadcast_to(np.asarray(null_mask, dtype=np.uint32), (n,)).copy()
    Ka = np.broadcast_to(np.asarray(K, dtype=np.int32), (n,)).copy()
    return TileSet(d, axis, idx, hw, nm, Ka)


def null_mask_of_boxes(c: np.ndarray, h: np.ndarray, one_arm: bool) -> np.ndarray:
    """Bit j-1 set when the open box (c - h, c + h) meets H_j.

    one-arm: H_1 = {theta <= 0}.  Multi-arm: H_j = {theta_j <= theta_0}; the open
    box meets it iff  c_j - h_j < c_0 + h_0.
    """
    # boxes that only touch a hypothesis' boundary (lattice neighbours, equal up to
    # rounding of the centres) do not meet its interior: compare with a margin
    eps = 1e-9 * np.max(h, axis=1)
    if one_arm:
        return ((c[:, 0] - h[:, 0]) < -eps).astype(np.uint32)
    m = np.zeros(c.shape[0], dtype=np.uint32)
    for j in range(1, c.shape[1]):
        meets = (c[:, j] - h[:, j]) - (c[:, 0] + h[:, 0]) < -eps
        m |= meets.astype(np.uint32) << np.uint32(j - 1)
    return m


def null_mask_basket(c: np.ndarray, h: np.ndarray, tnull) -> np.ndarray:
    """Basket design: bit i set when the open box (c - h, c + h) meets
    H_i = {theta_i <= t_i} (arm i's response rate at most its null rate)."""
    eps = 1e-9 * np.max(h, axis=1)
    m = np.zeros(c.shape[0], dtype=np.uint32)
    for i in range(c.shape[1]):
        meets = (c[:, i] - h[:, i]) - tnull[i] < -eps
        m |= meets.astype(np.uint32) << np.uint32(i)
    return m


# ----------------------------------------------------------------------------
# Designs
# ----------------------------------------------------------------------------
ONE_ARM = Design("one_arm_z_n50", "one_arm_z", 1, (50,))
TWO_ARM = Design("two_arm_pooled_z_n100", "two_arm_pooled_z", 2, (100,))
BAYES4 = Design("bayes4_looks_10_20_40", "bayes4", 4, (10, 20, 40))
# Basket trial of Sec. 10.1 (n = 35 per arm, one analysis, reject arm i when
# P(p_i > p_0i | data) > 85%).  The paper does not give the arms' null rates;
# these are a synthetic stand-in.
BERRY_P0 = (0.10, 0.15, 0.20, 0.25)
BERRY4 = Design("berry4_n35", "berry4", 4, (35,),
                arm_null=tuple(float(np.log(p / (1.0 - p))) for p in BERRY_P0))
BERRY_LAMBDA = 0.15


def lattice(lo: float, hi: float, cells: int) -> np.ndarray:
    h = (hi - lo) / (2.0 * cells)
    return lo + h * (2.0 * np.arange(cells) + 1.0)


# ----------------------------------------------------------------------------
# Tile sets
# ----------------------------------------------------------------------------
def one_arm_tiles(n_tiles: int = 64, K: int = 8192, lo: float = -2.0, hi: float = 0.0) -> TileSet:
    """1-D grid of equal half-width tiles over [lo, hi] (z-test validation shape)."""
    c = lattice(lo, hi, n_tiles)[:, None]
    h = np.full_like(c, (hi - lo) / (2.0 * n_tiles))
    nm = null_mask_of_boxes(c, h, one_arm=True)
    keep = nm != 0
    return from_centers(c[keep], h[keep], nm[keep], K)


def two_arm_grid(cells: int = 256, K: int = 16384, lo: float = -2.0, hi: float = 2.0) -> TileSet:
    """cells x cells grid over [lo, hi]^2; keeps boxes meeting theta_1 <= theta_0."""
    ax = lattice(lo, hi, cells)
    h = (hi - lo) / (2.0 * cells)
    j0, j1 = np.meshgrid(np.arange(cells), np.arange(cells), indexing="ij")
    j0, j1 = j0.ravel(), j1.ravel()
    c = np.stack([ax[j0], ax[j1]], axis=1)
    hw = np.full_like(c, h)
    nm = null_mask_of_boxes(c, hw, one_arm=False)
    keep = nm != 0
    idx = np.stack([j0[keep], j1[keep]], axis=1).astype(np.int32)
    return TileSet(2, [ax.copy(), ax.copy()], idx, hw[keep], nm[keep],
                   np.full(int(keep.sum()), K, dtype=np.int32))


def two_arm_adaptive(n_tiles: int = 1 << 18, seed: int = 1, levels=(4, 5, 6, 7),
                     log2K=(12, 13, 14, 15, 16), lo: float = -2.0, hi: float = 2.0) -> TileSet:
    """Throughput batch of mixed-level tiles (half-width 2^-l) with mixed K.

    Each tile draws its level and log2 K uniformly, then a centre uniformly on
    the level's lattice lo + h (2m + 1) inside [lo, hi]^2, redrawn until the open
    box meets theta_1 <= theta_0.  numpy PCG64 seeded with `seed`.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lev = rng.choice(np.asarray(levels), size=n_tiles)
    lk = rng.choice(np.asarray(log2K), size=n_tiles)
    h = 2.0 ** (-lev.astype(np.float64))
    cells = np.round((hi - lo) / (2.0 * h)).astype(np.int64)
    m0 = np.zeros(n_tiles, dtype=np.int64)
    m1 = np.zeros(n_tiles, dtype=np.int64)
    todo = np.arange(n_tiles)
    while todo.size:
        m0[todo] = rng.integers(0, cells[todo])
        m1[todo] = rng.integers(0, cells[todo])
        c0 = lo + h[todo] * (2.0 * m0[todo] + 1.0)
        c1 = lo + h[todo] * (2.0 * m1[todo] + 1.0)
        ok = (c1 - h[todo]) < (c0 + h[todo])
        todo = todo[~ok]
    c = np.stack([lo + h * (2.0 * m0 + 1.0), lo + h * (2.0 * m1 + 1.0)], axis=1)
    hw = np.stack([h, h], axis=1)
    nm = null_mask_of_boxes(c, hw, one_arm=False)
    K = (1 << lk).astype(np.int32)
    return from_centers(c, hw, nm, K)


LOGIT_LO = float(np.log(0.27 / 0.73))
LOGIT_HI = float(np.log(0.76 / 0.24))


def four_arm_grid(cells: int = 16, K: int = 1 << 14, lo: float = LOGIT_LO,
                  hi: float = LOGIT_HI) -> TileSet:
    """cells^4 grid over [lo, hi]^4 keeping boxes that meet at least one H_i."""
    ax = lattice(lo, hi, cells)
    h = (hi - lo) / (2.0 * cells)
    J = np.stack(np.meshgrid(*([np.arange(cells)] * 4), indexing="ij"), axis=-1).reshape(-1, 4)
    c = ax[J]
    hw = np.full_like(c, h)
    nm = null_mask_of_boxes(c, hw, one_arm=False)
    keep = nm != 0
    return TileSet(4, [ax.copy() for _ in range(4)], J[keep].astype(np.int32), hw[keep],
                   nm[keep], np.full(int(keep.sum()), K, dtype=np.int32))


def four_arm_refined(target: int = 1 << 20, K: int = 1 << 16, cells: int = 16,
                     max_level: int = 3, seed: int = 0) -> TileSet:
    """Adaptive refinement of the 4-arm platten.

    Start from the cells^4 null tiles; repeatedly split the tile of highest
    priority (smallest min_i |c_i - c_0|, i.e. nearest a null boundary; ties
    broken by a seeded random key) into its 16 children (each axis halved),
    keeping the children that still meet a null hypothesis, up to `max_level`
    splits deep, until at least `target` tiles exist.
    """
    base = four_arm_grid(cells, K)
    rng = np.random.Generator(np.random.PCG64(seed))
    c = base.centers
    h = base.halfwidth[:, 0].copy()
    lev = np.zeros(c.shape[0], dtype=np.int64)
    n_alive = c.shape[0]

    def prio(cc):
        return np.min(np.abs(cc[:, 1:] - cc[:, :1]), axis=1)

    heap = list(zip(prio(c).tolist(), rng.random(c.shape[0]).tolist(), range(c.shape[0])))
    heapq.heapify(heap)
    total = c.shape[0]
    signs = np.array([[1.0 if (m >> a) & 1 else -1.0 for a in range(4)] for m in range(16)])
    flat_c = list(c)
    flat_h = list(h)
    flat_l = list(lev)
    alive = [True] * total
    while n_alive < target and heap:
        _, _, i = heapq.heappop(heap)
        if flat_l[i] >= max_level:
            continue
        hc = flat_h[i] * 0.5
        kids = flat_c[i][None, :] + signs * hc
        khw = np.full_like(kids, hc)
        km = null_mask_of_boxes(kids, khw, one_arm=False)
        kids = kids[km != 0]
        alive[i] = False
        n_alive -= 1
        pk = prio(kids)
        rk = rng.random(kids.shape[0])
        for j in range(kids.shape[0]):
            flat_c.append(kids[j])
            flat_h.append(hc)
            flat_l.append(flat_l[i] + 1)
            alive.append(True)
            heapq.heappush(heap, (float(pk[j]), float(rk[j]), len(flat_c) - 1))
            n_alive += 1
    keep = np.nonzero(np.asarray(alive))[0]
    cc = np.stack([flat_c[i] for i in keep])
    hh = np.asarray([flat_h[i] for i in keep])
    hw = np.repeat(hh[:, None], 4, axis=1)
    nm = null_mask_of_boxes(cc, hw, one_arm=False)
    return from_centers(cc, hw, nm, K)


def berry_grid(cells: int = 16, K: int = 1 << 14, lo: float = -3.5, hi: float = 1.0,
               design: "Design" = None) -> TileSet:
    """cells^4 grid of the basket design over [lo, hi]^4 (logit p; the paper's
    figure of Sec. 10.1 spans theta_i in [-3.5, 1]), keeping boxes that meet at
    least one arm's null set."""
    design = design or BERRY4
    ax = lattice(lo, hi, cells)
    h = (hi - lo) / (2.0 * cells)
    J = np.stack(np.meshgrid(*([np.arange(cells)] * 4), indexing="ij"), axis=-1).reshape(-1, 4)
    c = ax[J]
    hw = np.full_like(c, h)
    nm = null_mask_basket(c, hw, design.arm_null)
    keep = nm != 0
    return TileSet(4, [ax.copy() for _ in range(4)], J[keep].astype(np.int32), hw[keep],
                   nm[keep], np.full(int(keep.sum()), K, dtype=np.int32))


CONFIGS = {
    "c1": lambda: (ONE_ARM, one_arm_tiles(64, 8192)),
    "c2": lambda: (TWO_ARM, two_arm_grid(256, 16384)),
    "c3": lambda: (TWO_ARM, two_arm_adaptive(1 << 18)),
    "c4": lambda: (BAYES4, four_arm_grid(16, 1 << 14)),
    "c5": lambda: (BAYES4, four_arm_refined(1 << 20, 1 << 16)),
    "berry": lambda: (BERRY4, berry_grid(16, 1 << 14)),
}
