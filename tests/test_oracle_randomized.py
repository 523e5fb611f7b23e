"""Pins of the oracle's randomised test (Sec. 7: the statistic (S, w) with an
independent uniform w, the threshold (lambda, c), compared lexicographically).

- The tie-break words are uniform (chi-square) and not the patients' draws.
- The per-tile threshold is the k-th smallest (S, w) pair: checked against a
  lexicographic sort of the exported statistics and words (numpy lexsort, not
  the oracle's qsort), and the calibrated pair rejects exactly k - 1 of the
  tile's own sims.
- c = 0 is the plain rule S < lambda.
- Thm. calibration with a continuous statistic: the mean of f at the
  randomised threshold equals floor((N+1) alpha)/(N+1) (two-sided, 3 sigma),
  where the plain threshold of the same discrete statistic falls short of it
  by the expected jump E[f_+ - f] at the threshold.
"""
import math

import numpy as np
from scipy import stats

from oracle import oracle as O
from paper_2212_10042_gb300 import workloads as W


def test_tiebreak_words_uniform_and_distinct():
    seed = 1234
    w = np.array([O.tiebreak(seed, k) for k in range(40000)], dtype=np.uint64)
    counts = np.bincount((w >> np.uint64(28)).astype(np.int64), minlength=16)
    chi2 = ((counts - len(w) / 16) ** 2 / (len(w) / 16)).sum()
    assert stats.chi2.sf(chi2, 15) > 1e-4
    u = np.array([O.uniform(seed, k, 0, 0) for k in range(2000)], dtype=np.uint64)
    assert np.mean(u == w[:2000]) < 0.01


def test_k_th_pair_by_lexsort_and_exact_rejections():
    tiles = W.one_arm_tiles(6, 700, lo=-0.6, hi=0.0)
    design = W.ONE_ARM
    cal = O.calibrate_rand(design, tiles, 0.025)
    sim = O.simulate(design, tiles, 0.0, want_S=True)
    w = np.array([O.tiebreak(design.seed, k) for k in range(700)], dtype=np.uint64)
    for i in range(tiles.n_tiles):
        Si = sim["S"][i]
        order = np.lexsort((w, Si))                      # primary key S, then w
        k = int(cal["k"][i])
        assert k >= 1
        assert cal["lambda_tile"][i] == Si[order[k - 1]]
        assert int(cal["c_tile"][i]) == int(w[order[k - 1]])
        R = O.simulate_rand(design, tiles.subset([i]), cal["lambda_tile"][i], int(cal["c_tile"][i]))["R"][0]
        assert R == k - 1
    # the global threshold is the lexicographic minimum of the tiles'
    pairs = sorted(zip(cal["lambda_tile"], cal["c_tile"].astype(np.int64)))
    assert (cal["lam"], cal["c"]) == (pairs[0][0], int(pairs[0][1]))


def test_c_zero_is_the_plain_rule():
    tiles = W.one_arm_tiles(8, 900, lo=-0.5, hi=0.2)
    for lam in (-1.9798989295959473, -1.5):
        a = O.simulate(W.ONE_ARM, tiles, lam)["R"]
        b = O.simulate_rand(W.ONE_ARM, tiles, lam, 0)["R"]
        assert np.array_equal(a, b)


def _f_rand(theta, lam, c):
    """exact P((S, w) < (lam, c)) for the n = 50 one-arm z-test (quantised p = t/2^32)."""
    p = O.threshold(theta) / 2.0 ** 32
    x = np.arange(51)
    S = np.array([O.stat_one_arm(int(v), 50) for v in x])
    pmf = stats.binom.pmf(x, 50, p)
    return float((pmf * (S < lam)).sum() + (pmf * (S == lam)).sum() * (c / 2.0 ** 32))


def test_randomised_calibration_is_tight():
    # N = 999, alpha = 0.0255 on a (near) point tile: k = floor(1000 alpha') = 25
    N, seeds, theta = 999, 300, -0.1
    tiles = W.from_centers([[theta]], 1e-9, 1, N)
    fr, fp = [], []
    for s in range(seeds):
        D = W.Design("one_arm", "one_arm_z", 1, (50,), seed=70000 + s)
        cal = O.calibrate_rand(D, tiles, 0.0255)
        assert cal["k"][0] == 25
        fr.append(_f_rand(theta, cal["lambda_tile"][0], int(cal["c_tile"][0])))
        fp.append(_f_rand(theta, cal["lambda_tile"][0], 0))           # the plain threshold
    fr, fp = np.asarray(fr), np.asarray(fp)
    target = 25 / 1000
    se = fr.std() / math.sqrt(seeds)
    assert abs(fr.mean() - target) <= 3 * se
    # the plain rule at the same order statistic sits below by the jump
    assert fp.mean() < target - 3 * fp.std() / math.sqrt(seeds)
