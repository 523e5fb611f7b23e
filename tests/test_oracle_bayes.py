"""Pins of the oracle's four-arm Bayesian design (Sec. 10.1 model, Sec. 10.2 design).

The posterior is checked against an independent dense-linear-algebra evaluation
of the same model (explicit 4x4 covariances, Gaussian conditioning, multivariate
normal marginal likelihood); the design's drop/freeze logic against hand-built
count paths; and the simulation against exact enumeration of a tiny variant.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2212_10042_gb300 import workloads as W

MU0, TAU2, IGA, IGB = -1.34, 100.0, 0.0005, 0.000005


def _posterior_linalg(x, n):
    x = np.asarray(x, float)
    n = np.asarray(n, float)
    th = np.log((x + 0.5) / (n - x + 0.5))
    s2 = 1 / (x + 0.5) + 1 / (n - x + 0.5)
    L = np.linspace(math.log(1e-6), math.log(1e3), 16)
    logw = np.zeros(16)
    pij = np.zeros((16, 3))
    one = np.ones(4)
    for j, l in enumerate(L):
        sig2 = math.exp(l)
        C_th = sig2 * np.eye(4) + TAU2 * np.outer(one, one)      # Cov(theta)
        C_obs = C_th + np.diag(s2)                                # Cov(theta_hat)
        logw[j] = (math.log(0.5) if j in (0, 15) else 0.0) \
            + stats.invgamma.logpdf(sig2, IGA, scale=IGB) + l \
            + stats.multivariate_normal.logpdf(th, MU0 * one, C_obs)
        K = np.linalg.solve(C_obs, C_th).T                         # C_th C_obs^-1
        mean = MU0 + K @ (th - MU0)
        cov = C_th - K @ C_th
        for i in range(1, 4):
            e = np.zeros(4)
            e[i], e[0] = 1, -1
            pij[j, i - 1] = stats.norm.cdf((e @ mean) / math.sqrt(e @ cov @ e))
    w = np.exp(logw - logw.max())
    w /= w.sum()
    return w @ pij


@pytest.mark.parametrize("x,n", [([3, 5, 2, 7], [10] * 4), ([12, 20, 9, 15], [40, 40, 20, 40]),
                                 ([0, 10, 10, 1], [10] * 4), ([20, 31, 17, 25], [40] * 4),
                                 ([5, 1, 9, 6], [10, 10, 20, 20])])
def test_posterior_matches_dense_linear_algebra(x, n):
    P = O.bayes4_posterior(x, n)
    ref = _posterior_linalg(x, n)
    assert np.allclose(P, ref, rtol=1e-10, atol=1e-13)


def test_posterior_symmetries():
    # identical data for arm i and control gives 1/2; permuting treatments permutes P
    P = O.bayes4_posterior([7, 7, 3, 9], [20] * 4)
    assert abs(P[0] - 0.5) < 1e-14
    a = O.bayes4_posterior([11, 4, 15, 8], [40] * 4)
    b = O.bayes4_posterior([11, 8, 4, 15], [40] * 4)
    assert np.allclose(a[[2, 0, 1]], b, rtol=0, atol=1e-15)
    # more successes on a treatment arm raise its posterior probability away from
    # the extreme counts (at x = 0 or n the empirical-logit variance is large and
    # the hierarchy shrinks the arm strongly, so P is not monotone there)
    ps = [O.bayes4_posterior([10, k, 10, 10], [40] * 4)[0] for k in range(4, 37, 4)]
    assert all(q > p for p, q in zip(ps, ps[1:]))


def test_design_drop_and_freeze():
    D = W.BAYES4
    # arm 1 is hopeless at look 1 -> dropped; its (x, n) = (0, 10) stays in the model
    xl = np.array([[7, 1, 10, 10], [13, 3, 17, 16], [25, 11, 30, 29]])
    P1 = O.bayes4_posterior(xl[0], [10] * 4)
    assert P1[0] < 0.1 and min(P1[1:]) >= 0.1
    P2 = O.bayes4_posterior([13, 1, 17, 16], [20, 10, 20, 20])
    assert all(p >= 0.1 for p in P2[1:])
    P3 = O.bayes4_posterior([25, 1, 30, 29], [40, 10, 40, 40])
    S_all = O.bayes4_stat(D, xl, 0b111)
    assert S_all == min(1 - P3[1], 1 - P3[2])
    # only arm 3 null: S uses arm 3 alone
    assert O.bayes4_stat(D, xl, 0b100) == 1 - P3[2]
    # only the dropped arm null: nothing to reject
    assert O.bayes4_stat(D, xl, 0b001) == math.inf
    # every treatment dropped at look 1 stops the trial
    assert O.bayes4_stat(D, np.array([[9, 0, 0, 0], [18, 1, 1, 1], [36, 2, 2, 2]]), 0b111) == math.inf


def test_tiny_design_simulation_matches_enumeration():
    # looks after 1, 2, 3 patients per arm: 2^3 outcome paths per arm, 8^4 in total
    D = W.Design("bayes4_tiny", "bayes4", 4, (1, 2, 3), drop=0.3)
    theta = np.array([0.1, 0.4, -0.2, 0.3])
    p = np.array([O.threshold(t) / 2.0 ** 32 for t in theta])
    lam = 0.5
    paths = list(itertools.product([0, 1], repeat=3))
    f = 0.0
    for combo in itertools.product(range(8), repeat=4):
        xl = np.zeros((3, 4), dtype=np.int32)
        pr = 1.0
        for a, pi in enumerate(combo):
            incs = paths[pi]
            xl[:, a] = np.cumsum(incs)
            pr *= np.prod([p[a] if s else 1 - p[a] for s in incs])
        if O.bayes4_stat(D, xl, 0b111) < lam:
            f += pr
    K = 40000
    tiles = W.from_centers([theta], 0.01, 0b111, K)
    R = O.simulate(D, tiles, lam)["R"][0]
    assert 0.02 < f < 0.98
    assert abs(R / K - f) <= 4.5 * math.sqrt(f * (1 - f) / K)
