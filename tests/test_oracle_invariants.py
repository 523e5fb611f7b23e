"""Statistical invariants of the oracle's procedures over many seeds.

- Validation (Alg. validation): the tile bound is at least the exact worst-case
  Type I Error on the tile with probability >= 1 - delta (Sec. 6.2).
- Pointwise calibration (Thm. calibration): E f(lambda_hat) <= floor((N+1)a)/(N+1).
- Global calibration (Alg. calibration): E f_{lambda*}(theta) <= alpha on the
  null region (checked at the boundary point, where f is largest).
"""
import math

import numpy as np
from scipy import stats

from oracle import oracle as O
from paper_2212_10042_gb300 import workloads as W


def _f_one_arm(theta, lam):
    """exact P_theta(S(X) < lam) for the n = 50 one-arm z-test (quantised p = t/2^32)."""
    p = O.threshold(theta) / 2.0 ** 32
    x = np.arange(51)
    S = np.array([O.stat_one_arm(int(v), 50) for v in x])
    return float((stats.binom.pmf(x, 50, p) * (S < lam)).sum())


def test_validation_coverage_over_seeds():
    delta, K, seeds = 0.01, 2048, 60
    base = W.one_arm_tiles(16, K, lo=-0.5, hi=0.0)
    c, h = base.centers[:, 0], base.halfwidth[:, 0]
    worst = np.array([_f_one_arm(ci + hi, -1.96) for ci, hi in zip(c, h)])  # f increasing in theta
    fails = np.zeros(len(c), dtype=int)
    for s in range(seeds):
        D = W.Design("one_arm", "one_arm_z", 1, (50,), seed=1000 + s)
        R = O.simulate(D, base, -1.96)["R"]
        b = O.validate_bounds(D, base, R, delta)["bound"]
        fails += b < worst
    # each tile fails with probability <= delta: allow a 3-sigma band per tile
    assert fails.max() <= delta * seeds + 3 * math.sqrt(delta * seeds) + 1
    assert fails.sum() <= delta * seeds * len(c) + 3 * math.sqrt(delta * seeds * len(c))


def test_pointwise_calibration_theorem():
    # N = 999, alpha = 0.0255 on a (near) point tile: k = floor(1000 alpha') = 25
    N, seeds, theta = 999, 300, -0.1
    tiles = W.from_centers([[theta]], 1e-9, 1, N)
    vals = []
    for s in range(seeds):
        D = W.Design("one_arm", "one_arm_z", 1, (50,), seed=50000 + s)
        cal = O.calibrate(D, tiles, 0.0255)
        assert cal["k"][0] == 25
        vals.append(_f_one_arm(theta, cal["lambda_tile"][0]))
    vals = np.asarray(vals)
    bound = 25 / 1000
    assert vals.mean() <= bound + 3 * vals.std() / math.sqrt(seeds)


def test_global_calibration_controls_level():
    alpha, K, seeds = 0.025, 1000, 120
    tiles = W.one_arm_tiles(8, K, lo=-0.5, hi=0.0)
    vals = []
    for s in range(seeds):
        D = W.Design("one_arm", "one_arm_z", 1, (50,), seed=90000 + s)
        cal = O.calibrate(D, tiles, alpha)
        assert cal["lam"] == cal["lambda_tile"].min()
        vals.append(_f_one_arm(0.0, cal["lam"]))
    vals = np.asarray(vals)
    assert vals.mean() <= alpha + 3 * vals.std() / math.sqrt(seeds)
