"""Pins of the oracle's random numbers, Bernoulli draws, statistics and sims.

Each check ties the oracle to something other than itself: published
known-answer vectors, exact binomial laws (scipy), FP64 closed forms, and the
exact Type I Error / derivative of the one- and two-arm tests.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2212_10042_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(x, 16) for x in line.split()]
                rows.append((v[:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert list(O.philox(ctr, key)) == expect


def test_uniform_layout_and_uniformity():
    # word j of sim k, arm a is word j%4 of Philox(ctr=(k, a, j//4, 0), key=seed)
    seed = (7 << 32) | 3
    w = O.philox([5, 1, 2, 0], [3, 7])
    assert [O.uniform(seed, 5, 1, 8 + i) for i in range(4)] == list(w)
    # chi-square uniformity of the top byte over 2^15 words
    u = np.array([O.uniform(0, k, a, j) for k in range(64) for a in range(4) for j in range(128)],
                 dtype=np.uint64)
    counts = np.bincount((u >> np.uint64(24)).astype(np.int64), minlength=256)
    chi2 = ((counts - counts.mean()) ** 2 / counts.mean()).sum()
    assert stats.chi2.sf(chi2, 255) > 1e-4


def test_threshold_definition():
    assert O.threshold(0.0) == 1 << 31
    for th in np.linspace(-6, 6, 97):
        p = 1.0 / (1.0 + math.exp(-th))
        t = O.threshold(th)
        assert abs(t / 2.0 ** 32 - p) <= 2.0 ** -32
    assert O.threshold(60.0) == 2 ** 32 - 1
    assert O.threshold(-800.0) == 0


def test_count_law_is_binomial():
    # counts of n=50 draws at p = t/2^32 follow Binom(50, p): chi-square over 4096 sims
    D = W.ONE_ARM
    th = -0.4
    p = O.threshold(th) / 2.0 ** 32
    xs = np.array([O.counts(D, [th], k)[0, 0] for k in range(4096)])
    obs = np.bincount(xs, minlength=51)
    exp = stats.binom.pmf(np.arange(51), 50, p) * len(xs)
    lo, hi = 8, 35
    o = np.concatenate([[obs[:lo].sum()], obs[lo:hi], [obs[hi:].sum()]])
    e = np.concatenate([[exp[:lo].sum()], exp[lo:hi], [exp[hi:].sum()]])
    chi2 = ((o - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi2, len(o) - 1) > 1e-4
    # looks are nested prefixes of the same patients
    D4 = W.BAYES4
    x = O.counts(D4, [0.1, -0.3, 0.5, 0.0], 17)
    assert np.all(np.diff(x, axis=0) >= 0) and np.all(x[0] <= 10) and np.all(x[-1] <= 40)


def test_one_arm_statistic():
    # S = -z with z = (x - 25) / sqrt(12.5); reject at lambda = -1.96 iff x >= 32
    for x in range(51):
        z = (x - 25.0) / math.sqrt(12.5)
        S = O.stat_one_arm(x, 50, 0.5)
        assert abs(S + z) <= 1e-6 * max(1.0, abs(z))
        assert (S < -1.96) == (x >= 32)
    assert abs(O.stat_one_arm(31, 50) + 1.697056) < 1e-6
    assert abs(O.stat_one_arm(32, 50) + 1.979899) < 1e-6


def test_two_arm_statistic_against_fp64():
    n = 100
    x0, x1 = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    pb = (x0 + x1) / (2.0 * n)
    var = pb * (1 - pb) * (2.0 / n)
    with np.errstate(divide="ignore", invalid="ignore"):
        z64 = np.where(var > 0, (x1 / n - x0 / n) / np.sqrt(var), 0.0)
    S = np.array([[O.stat_two_arm(a, b, n, n) for b in range(n + 1)] for a in range(n + 1)])
    assert np.all(np.abs(S + z64) <= 4e-6 * np.maximum(1.0, np.abs(z64)))  # a few FP32 ulps
    # FP32 and FP64 take the same decision at z > 1.96 on every cell
    assert np.array_equal(S < -1.96, z64 > 1.96)
    # antisymmetry in (x0, x1), zero on the degenerate cells
    assert np.array_equal(S, -S.T)
    assert S[0, 0] == 0.0 and S[n, n] == 0.0
    # rejection is monotone: more treatment successes never un-reject
    rej = S < -1.96
    assert np.all(rej[:, 1:] >= rej[:, :-1]) and np.all(rej[:-1, :] >= rej[1:, :])


def _one_arm_exact(theta):
    p = O.threshold(theta) / 2.0 ** 32
    f = stats.binom.sf(31, 50, p)
    df = 50 * math.comb(49, 31) * p ** 32 * (1 - p) ** 19
    return f, df


def test_one_arm_exact_pins():
    # exact Type I Error of the one-arm test and its theta-derivative
    f, df = _one_arm_exact(0.0)
    assert abs(f - 3.245432353613609e-2) < 1e-15
    assert abs(df - 2.565560760640295e-1) < 1e-14
    # derivative identity: d/dtheta P(X >= 32) = E[1{X>=32} (X - n p)]
    p = O.threshold(-0.3) / 2.0 ** 32
    x = np.arange(51)
    score = (stats.binom.pmf(x, 50, p) * (x >= 32) * (x - 50 * p)).sum()
    assert abs(score - _one_arm_exact(-0.3)[1]) < 1e-15


@pytest.mark.parametrize("theta", [0.0, -0.25, -0.5])
def test_one_arm_mc_matches_exact(theta):
    K = 20000
    tiles = W.from_centers([[theta]], 1 / 64, 1, K)
    out = O.simulate(W.ONE_ARM, tiles, -1.96)
    f, df = _one_arm_exact(theta)
    R = out["R"][0]
    assert abs(R / K - f) <= 4.5 * math.sqrt(f * (1 - f) / K) + 1e-12
    # score-function gradient estimate G/K against the exact derivative
    p = O.threshold(theta) / 2.0 ** 32
    x = np.arange(51)
    pm = stats.binom.pmf(x, 50, p)
    g = (x >= 32) * (x - 50 * p)
    sd = math.sqrt(((g ** 2 * pm).sum() - df ** 2) / K)
    assert abs(out["score"][0, 0] / K - df) <= 4.5 * sd + 1e-12
    # score = Xrej - n sigmoid(theta) R (grad A uses the model's p, not t/2^32)
    sig = 1 / (1 + math.exp(-theta))
    assert abs(out["score"][0, 0] - (out["Xrej"][0, 0] - 50 * sig * R)) < 1e-9


def _two_arm_exact(th0, th1, lam=-1.96):
    n = 100
    p0 = O.threshold(th0) / 2.0 ** 32
    p1 = O.threshold(th1) / 2.0 ** 32
    x = np.arange(n + 1)
    S = np.array([[O.stat_two_arm(a, b, n, n) for b in x] for a in x])
    rej = (S < lam).astype(float)
    P = np.outer(stats.binom.pmf(x, n, p0), stats.binom.pmf(x, n, p1))
    f = (P * rej).sum()
    g0 = (P * rej * (x[:, None] - n * p0)).sum()
    g1 = (P * rej * (x[None, :] - n * p1)).sum()
    return f, np.array([g0, g1])


def test_two_arm_exact_pins_and_mc():
    f, g = _two_arm_exact(0.0, 0.0)
    assert abs(f - 0.0279828802) < 5e-10
    assert np.allclose(g, [-0.2269818864, 0.2269818864], atol=5e-10)
    assert abs(_two_arm_exact(-1.0, -1.0)[0] - 0.0248004191) < 5e-10
    assert abs(_two_arm_exact(2.0, 2.0)[0] - 0.0256140821) < 5e-10
    K = 12000
    th = [0.1, -0.05]
    tiles = W.from_centers([th], 1 / 128, 1, K)
    out = O.simulate(W.TWO_ARM, tiles, -1.96)
    f, g = _two_arm_exact(*th)
    assert abs(out["R"][0] / K - f) <= 4.5 * math.sqrt(f * (1 - f) / K)
    # gradient: |G/K - grad f| within a loose MC band (|T - nP| <= 100)
    assert np.all(np.abs(out["score"][0] / K - g) <= 4.5 * 100 * math.sqrt(f / K))


def test_crn_shared_across_tiles():
    # two tiles at the same centre see identical sims (common random numbers),
    # and a prefix K gives the prefix of the same sims
    tiles = W.from_centers([[-0.1], [-0.1]], 1 / 64, 1, [3000, 1000])
    S = O.simulate(W.ONE_ARM, tiles, -1.96, want_S=True)["S"]
    assert np.array_equal(S[0][:1000], S[1])
