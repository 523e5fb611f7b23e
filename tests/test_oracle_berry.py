"""Pins of the oracle's basket design (Sec. 10.1, Bayesian basket trial).

- The posterior P(theta_i > 0 | x) against dense linear algebra: for every
  node of s2 the joint Gaussian of the offset log-odds (prior covariance
  s2 I + 100 11', likelihood N(theta_hat, diag s_i^2)) conditioned by matrix
  inversion, the node weights from the multivariate normal density of theta_hat;
  the oracle uses the scalar rank-one formulas instead.
- Monotone in the arm's own successes away from x = 0 and x = n, decreasing
  in its null rate, and
  arm-permutation symmetric when the null rates are equal.
- A tiny basket (n = 4 per arm: 5^4 outcomes) by exact enumeration against the
  oracle's simulation (counts, statistic and rejection plumbing).
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2212_10042_gb300 import workloads as W

MU0, TAU2, IGA, IGB, NODES = -1.34, 100.0, 0.0005, 0.000005, 16


def _dense_posterior(x, n, tnull):
    x = np.asarray(x, dtype=float)
    xs, fs = x + 0.5, n - x + 0.5
    th = np.log(xs / fs) - np.asarray(tnull)
    s2 = 1.0 / xs + 1.0 / fs
    Ls = np.linspace(math.log(1e-6), math.log(1e3), NODES)
    logw, Pj = [], []
    one = np.ones(4)
    for j, L in enumerate(Ls):
        sig2 = math.exp(L)
        Sigma = sig2 * np.eye(4) + TAU2 * np.outer(one, one)
        C = Sigma + np.diag(s2)
        r = th - MU0
        _, logdet = np.linalg.slogdet(C)
        quad = r @ np.linalg.solve(C, r)
        trap = math.log(0.5) if j in (0, NODES - 1) else 0.0
        # node weight: IG prior density x Jacobian s2, times N(theta_hat; mu0, C) up to constants
        logw.append(trap - (IGA + 1.0) * L - IGB / sig2 + L - 0.5 * logdet - 0.5 * quad + 0.5 * math.log(TAU2))
        G = Sigma @ np.linalg.inv(C)
        mean = MU0 * one + G @ r
        cov = Sigma - G @ Sigma
        Pj.append(stats.norm.cdf(mean / np.sqrt(np.diag(cov))))
    logw = np.array(logw)
    w = np.exp(logw - logw.max())
    return (w[:, None] * np.array(Pj)).sum(0) / w.sum()


def test_posterior_against_dense_linear_algebra():
    rng = np.random.default_rng(3)
    tnull = W.BERRY4.arm_null
    for _ in range(40):
        x = rng.integers(0, 36, size=4)
        P = O.berry_posterior(x, 35, tnull)
        Q = _dense_posterior(x, 35, tnull)
        assert np.allclose(P, Q, rtol=1e-9, atol=1e-13), (x, P, Q)


def test_posterior_monotone_and_symmetric():
    tnull = W.BERRY4.arm_null
    base = np.array([8, 9, 10, 11])
    # Strictly increasing in the interior. At x = 0 and x = n the approximate
    # likelihood's variance 1/(x+1/2) + 1/(n-x+1/2) is large and the arm shrinks
    # towards the pooled mean, so the posterior turns back there (checked too).
    prev = -1.0
    for x0 in range(1, 22):
        P = O.berry_posterior([x0, 9, 10, 11], 35, tnull)
        assert P[0] > prev, x0
        prev = P[0]
    ends = [O.berry_posterior([x0, 9, 10, 11], 35, tnull)[0] for x0 in (0, 1, 34, 35)]
    assert ends[0] > ends[1] and ends[3] < ends[2]
    lo = O.berry_posterior(base, 35, (-2.0, -1.5, -1.5, -1.5))[0]
    hi = O.berry_posterior(base, 35, (-1.0, -1.5, -1.5, -1.5))[0]
    assert hi < lo      # a higher null rate is harder to beat
    eq = (-1.5,) * 4
    P = O.berry_posterior([3, 7, 12, 20], 35, eq)
    Pp = O.berry_posterior([20, 3, 12, 7], 35, eq)
    assert np.allclose(Pp, P[[3, 0, 2, 1]], rtol=1e-14, atol=0)


@pytest.mark.parametrize("theta", [(-1.9, -1.9, -1.5, -1.2), (-2.4, -1.0, -1.3, -0.9)])
def test_tiny_basket_exact_fwer_against_simulation(theta):
    design = W.Design("berry4_n4", "berry4", 4, (4,), seed=11, arm_null=W.BERRY4.arm_null)
    c = np.array([theta])
    h = np.full_like(c, 1e-9)
    nm = W.null_mask_basket(c, h, design.arm_null)
    assert nm[0] != 0
    tiles = W.from_centers(c, h, nm, 40000)
    # exact P(S < lambda) over the 5^4 outcomes with the simulation's p = t / 2^32
    p = [O.threshold(t) / 2.0 ** 32 for t in theta]
    pm = [stats.binom.pmf(np.arange(5), 4, pi) for pi in p]
    exact = 0.0
    for x in np.ndindex(5, 5, 5, 5):
        if O.berry_stat(design, np.array(x), int(nm[0])) < W.BERRY_LAMBDA:
            exact += pm[0][x[0]] * pm[1][x[1]] * pm[2][x[2]] * pm[3][x[3]]
    R = O.simulate(design, tiles, W.BERRY_LAMBDA)["R"][0]
    K = 40000
    sd = math.sqrt(max(exact * (1 - exact), 1e-12) / K)
    assert abs(R / K - exact) <= 4.5 * sd + 1e-12
    assert 0.005 < exact < 0.995   # neither never nor always: the check is not vacuous
