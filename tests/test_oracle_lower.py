"""Pins of the oracle's lower bounds (Rem. extension-lower).

- Lower Clopper-Pearson l = Beta^{-1}(delta; R, K-R+1): the closed forms at
  R = 1 (1 - (1-delta)^{1/K}) and R = K (delta^{1/K}), scipy's beta quantile,
  and the binomial symmetry l(R, K) = 1 - u(K-R, K) against the upper bound
  (its own CDF sum, not the tail sum the lower bound uses).
- The lower Tilt-Bound, applied to the exact value of f at the centre, is below
  the exact f everywhere in the box (one-arm z-test by the binomial law, two-arm
  pooled z-test by enumeration of its 101^2 cells): the inequality of the
  remark, which a dropped term, a wrong sign or the wrong a would break.
- Its limits: l at the centre of a vanishing box (q* -> infinity), 0 for l = 0,
  non-decreasing in l and non-increasing in the box size (strictly where it is
  positive); and lower <= exact f <= upper on every tile.
- Coverage over seeds: the lower bound from simulated counts exceeds the least
  exact f on the box with probability <= delta.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2212_10042_gb300 import workloads as W


def _sig(t):
    return 1.0 / (1.0 + math.exp(-t))


def _f1(theta):
    """exact P(X >= 32), X ~ Binom(50, sigmoid(theta)): the one-arm z-test at lambda = -1.96."""
    return float(stats.binom.sf(31, 50, _sig(theta)))


def _f2_table():
    x = np.arange(101)
    S = np.array([[O.stat_two_arm(int(a), int(b), 100, 100) for b in x] for a in x])
    return x, S < -1.96


def _f2(theta, table):
    x, rej = table
    p0 = stats.binom.pmf(x, 100, _sig(theta[0]))
    p1 = stats.binom.pmf(x, 100, _sig(theta[1]))
    return float(p0 @ rej @ p1)


@pytest.mark.parametrize("N", [8192, 16384, 65536])
@pytest.mark.parametrize("delta", [0.01, 0.05])
def test_cp_lower_closed_forms(N, delta):
    assert O.cp_lower(0, N, delta) == 0.0
    r1 = -math.expm1(math.log1p(-delta) / N)
    assert abs(O.cp_lower(1, N, delta) - r1) <= 1e-13 * r1
    rN = math.exp(math.log(delta) / N)
    assert abs(O.cp_lower(N, N, delta) - rN) <= 1e-13 * rN


def test_cp_lower_scipy_and_symmetry():
    rng = np.random.default_rng(4)
    for N in [10, 50, 1000, 16384, 65536]:
        for R in sorted(set([1, 2, N // 3, N - 1, N] + list(rng.integers(1, N + 1, 5)))):
            for delta in [0.01, 0.05]:
                lo = O.cp_lower(R, N, delta)
                ref = stats.beta.ppf(delta, R, N - R + 1)
                assert abs(lo - ref) <= 2e-9 * ref
                if lo > 0.05:   # 1 - u(N-R) keeps 1e-16 absolute digits
                    up = O.cp_upper(N - R, N, delta)
                    assert abs(lo - (1.0 - up)) <= 1e-12 * lo


@pytest.mark.parametrize("theta0,h", [(-0.5, 1 / 64), (0.0, 1 / 64), (0.3, 1 / 8), (-1.0, 1 / 4), (0.8, 1 / 16)])
def test_lower_tilt_bound_below_exact_f_one_arm(theta0, h):
    f0 = _f1(theta0)
    low, q = O.tilt_lower([theta0], [h], f0, [50.0])
    grid = np.linspace(theta0 - h, theta0 + h, 401)
    fmin = min(_f1(t) for t in grid)
    assert 0.0 <= low <= fmin * (1 + 1e-12)
    assert q >= 1.0
    # and it is informative: within the box's own spread of f below the least value
    assert low >= fmin - (max(_f1(t) for t in grid) - fmin) * 4 - 1e-12


def test_lower_tilt_bound_below_exact_f_two_arm():
    table = _f2_table()
    for c, h in [((0.0, 0.0), 1 / 128), ((0.5, -0.5), 1 / 32), ((-1.0, -1.2), 1 / 16)]:
        f0 = _f2(c, table)
        low, _ = O.tilt_lower(list(c), [h, h], f0, [100.0, 100.0])
        pts = [(c[0] + a * h, c[1] + b * h) for a in np.linspace(-1, 1, 9) for b in np.linspace(-1, 1, 9)]
        fmin = min(_f2(p, table) for p in pts)
        assert 0.0 <= low <= fmin * (1 + 1e-12)


def test_lower_tilt_bound_limits_and_monotonicity():
    l = 0.03
    low, q = O.tilt_lower([0.1], [1e-9], l, [50.0])
    assert abs(low - l) <= 1e-6 * l and q > 1e3
    assert O.tilt_lower([0.1], [0.05], 0.0, [50.0])[0] == 0.0
    # non-decreasing in l, strictly once informative (small l on a wide box gives 0)
    vals = [O.tilt_lower([0.1], [0.05], x, [50.0])[0] for x in (0.001, 0.01, 0.03, 0.1, 0.5)]
    assert all(b >= a and (b > a or a == 0.0) for a, b in zip(vals, vals[1:])) and vals[-1] > 0
    sizes = [O.tilt_lower([0.1], [h], l, [50.0])[0] for h in (0.001, 0.01, 0.05, 0.2)]
    assert all(b <= a and (b < a or b == 0.0) for a, b in zip(sizes, sizes[1:])) and sizes[0] > 0
    # the lower bound is the complement of the upper bound of 1 - F taken in log form
    lb, _ = O.tilt_bound_log([0.1], [0.05], math.log1p(-l), [50.0])
    assert abs(O.tilt_lower([0.1], [0.05], l, [50.0])[0] - (-math.expm1(lb))) <= 1e-15


def test_band_brackets_exact_f():
    for theta0, h in [(-0.5, 1 / 32), (0.2, 1 / 8)]:
        f0 = _f1(theta0)
        low, _ = O.tilt_lower([theta0], [h], f0, [50.0])
        up, _ = O.tilt_bound([theta0], [h], f0, [50.0])
        grid = np.linspace(theta0 - h, theta0 + h, 201)
        fs = np.array([_f1(t) for t in grid])
        assert low <= fs.min() and fs.max() <= up


def test_lower_validation_coverage_over_seeds():
    delta, K, seeds = 0.05, 2048, 60
    base = W.one_arm_tiles(16, K, lo=-0.5, hi=0.0)
    c, h = base.centers[:, 0], base.halfwidth[:, 0]
    # the simulation's p is t/2^32; f is increasing in theta, least at the left edge
    least = np.array([float(stats.binom.sf(31, 50, O.threshold(ci - hi) / 2.0 ** 32)) for ci, hi in zip(c, h)])
    fails = np.zeros(len(c), dtype=int)
    for s in range(seeds):
        D = W.Design("one_arm", "one_arm_z", 1, (50,), seed=3000 + s)
        R = O.simulate(D, base, -1.96)["R"]
        low = O.validate_lower(D, base, R, delta)
        assert np.all(low["l0"] <= R / K + 1e-15)
        fails += low["lower"] > least
    assert fails.max() <= delta * seeds + 3 * math.sqrt(delta * seeds) + 1
    assert fails.sum() <= delta * seeds * len(c) + 3 * math.sqrt(delta * seeds * len(c))
