"""Pin of the oracle's plain calibration selection (Eq. calibrated-threshold,
Thm. calibration, Sec. 7): for every tile, lambda_i is the k_i-th smallest of
the tile's own simulated statistics, k_i = floor((K_i + 1) alpha'_i), 1-indexed,
and -inf when k_i = 0 (the tile never rejects).

The expected values come from numpy, not from the oracle's selection: the
statistics the oracle exports (`simulate(..., want_S=True)`) are sorted with
np.sort and indexed, and the index is recomputed from the oracle's alpha'
(pinned on its own in test_oracle_bounds.py).  Two further checks hold for
the k-th order statistic with ties and without sorting at all:
#{S < lambda_i} < k_i <= #{S <= lambda_i}.

The statistics here are discrete (51 values for one arm, a few thousand for two
arms), so neighbouring order statistics are often equal.  The tile sets are
chosen so that many tiles sit at the edge of a tie group
(S_(k-1) != S_(k) and S_(k) != S_(k+1)); the tests assert that such tiles exist,
so that selecting one position too low or too high fails.
"""
import math

import numpy as np

from oracle import oracle as O
from paper_2212_10042_gb300 import workloads as W


def _one_arm_ragged(n=240, seed=17):
    rng = np.random.default_rng(seed)
    c = np.linspace(-0.45, 0.25, n)[:, None]
    h = np.full_like(c, 0.01)
    K = rng.integers(40, 2500, size=n).astype(np.int32)
    K[:6] = [1, 2, 3, 39, 40, 41]          # k = 0 (never rejects) and the first k = 1 tiles
    nm = np.ones(n, dtype=np.uint32)
    return W.from_centers(c, h, nm, K)


def _two_arm_ragged(seed=5):
    base = W.two_arm_grid(10, 1, lo=-1.0, hi=1.0)
    rng = np.random.default_rng(seed)
    K = rng.integers(1, 1800, size=base.n_tiles).astype(np.int32)
    K[:3] = [1, 5, 40]
    return base.with_K(K)


def _check(design, tiles, alpha):
    cal = O.calibrate(design, tiles, alpha)
    S = O.simulate(design, tiles, 0.0, want_S=True)["S"]
    ap = cal["alpha_prime"]
    k_np = np.minimum(np.floor((tiles.K.astype(np.float64) + 1.0) * ap).astype(np.int64), tiles.K)
    assert np.array_equal(cal["k"], k_np)
    low_edge = high_edge = zero = 0
    for i in range(tiles.n_tiles):
        Si = np.asarray(S[i], dtype=np.float64)
        assert len(Si) == tiles.K[i]
        k = int(k_np[i])
        lam = cal["lambda_tile"][i]
        if k == 0:
            zero += 1
            assert lam == -math.inf
            continue
        srt = np.sort(Si, kind="stable")
        assert lam == srt[k - 1], (i, k)
        assert int((Si < lam).sum()) < k <= int((Si <= lam).sum()), (i, k)
        if k >= 2 and srt[k - 2] != srt[k - 1]:
            low_edge += 1
        if k < len(srt) and srt[k] != srt[k - 1]:
            high_edge += 1
    assert cal["lam"] == np.min(cal["lambda_tile"])
    return zero, low_edge, high_edge


def test_one_arm_selection_is_the_kth_order_statistic():
    zero, low_edge, high_edge = _check(W.ONE_ARM, _one_arm_ragged(), 0.025)
    assert zero >= 4                    # K_i = 1, 2, 3 and 39 give k_i = 0
    assert low_edge >= 10 and high_edge >= 10, (low_edge, high_edge)


def test_two_arm_selection_is_the_kth_order_statistic():
    zero, low_edge, high_edge = _check(W.TWO_ARM, _two_arm_ragged(), 0.05)
    assert zero >= 1
    assert low_edge >= 20 and high_edge >= 20, (low_edge, high_edge)


def test_selection_at_every_k_of_one_tile():
    """One tile, the same CRN prefix at every K from 1 to 400: each K gives its own
    k_i, and the selection follows the sorted prefix of the sims exactly (the
    index grows by one at each K where (K + 1) alpha' crosses an integer)."""
    c = np.full((400, 1), -0.05)
    h = np.full_like(c, 0.02)
    K = np.arange(1, 401, dtype=np.int32)
    tiles = W.from_centers(c, h, np.ones(400, dtype=np.uint32), K)
    cal = O.calibrate(W.ONE_ARM, tiles, 0.1)
    S_all = np.asarray(O.simulate(W.ONE_ARM, tiles.subset([399]), 0.0, want_S=True)["S"][0])
    ap = cal["alpha_prime"][0]
    assert np.all(cal["alpha_prime"] == ap)      # the same tile geometry throughout
    for j, Kj in enumerate(K):
        k = min(int(math.floor((Kj + 1.0) * ap)), int(Kj))
        want = -math.inf if k == 0 else float(np.sort(S_all[:Kj])[k - 1])
        assert cal["lambda_tile"][j] == want, (Kj, k)
