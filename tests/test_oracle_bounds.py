"""Pins of the oracle's Clopper-Pearson bound, Tilt-Bound and calibration target.

Against: scipy's Beta quantile and CP closed forms; the normal-location
Tilt-Bound closed forms (calculus on Eq. tilt-bound-normal) and the numbers the
paper prints for them; brute-force q grids; enumeration of psi from the
binomial law; a dense interior scan of the box (Thm. 3); and the duality between
the Tilt-Bound and its inverse (Eq. tilt-bound-inv).
"""
import math
import os

import numpy as np
import pytest
from scipy import special, stats

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_values():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_values.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


@pytest.mark.parametrize("R,N,delta", [(0, 8192, 0.01), (1, 8192, 0.01), (235, 8192, 0.01),
                                       (409, 16384, 0.01), (5000, 16384, 0.05), (16383, 16384, 0.01),
                                       (1638, 65536, 0.01), (3, 20, 0.2), (0, 1, 0.01)])
def test_clopper_pearson_against_scipy(R, N, delta):
    u = O.cp_upper(R, N, delta)
    ref = stats.beta.ppf(1 - delta, R + 1, N - R)
    assert abs(u - ref) <= 1e-13 * ref


def test_clopper_pearson_closed_forms():
    for N in (1, 50, 8192, 65536):
        for delta in (0.01, 0.05):
            assert abs(O.cp_upper(0, N, delta) - (-math.expm1(math.log(delta) / N))) <= 1e-14 * O.cp_upper(0, N, delta)
            assert abs(O.cp_upper(N - 1, N, delta) - (1 - delta) ** (1.0 / N)) <= 1e-14
            assert O.cp_upper(N, N, delta) == 1.0
    assert abs(O.cp_upper(0, 8192, 0.01) - 5.619965844467e-4) < 1e-15
    # monotone in R
    us = [O.cp_upper(r, 1000, 0.01) for r in range(0, 60)]
    assert all(b > a for a, b in zip(us, us[1:]))


def test_normal_tilt_bound_closed_form_and_paper_values():
    pv = _paper_values()
    # one-sided z-test at level 2.5%: f(theta) = Phi(theta - z_{0.975}); theta_0 = -0.25
    z = stats.norm.ppf(0.975)
    a = stats.norm.cdf(-0.25 - z)
    for v in (0.05, 0.1, 0.25, 0.4):
        b, q = O.tilt_bound([-0.25], [v], a, [1.0], family=O.FAMILY_NORMAL)
        # calculus on a^(1-1/q) exp((q-1) v^2/2): q* = sqrt(-2 log a)/|v|
        qs = math.sqrt(-2 * math.log(a)) / v
        us = a ** (1 - 1 / qs) * math.exp((qs - 1) * v * v / 2)
        assert abs(b - us) <= 1e-12 * us
        assert abs(q - qs) <= 1e-9 * qs
    b, _ = O.tilt_bound([-0.25], [0.25], a, [1.0], family=O.FAMILY_NORMAL)
    assert round(b, 4) == pv["normal_tilt_bound_v025"]
    assert round(stats.norm.cdf(0 - z), 3) == pv["normal_true_tie_v025"]
    assert round(b - stats.norm.cdf(-z), 4) == pv["normal_gap_at_zero"]


def test_normal_alpha_prime_closed_form():
    # M(q) = q/(q-1) log alpha - q v^2/2 is maximised at q* = 1 + sqrt(-2 log alpha)/|v|
    for alpha in (0.025, 0.05):
        for v in (0.01, 0.1, 0.3):
            ap, q = O.alpha_prime([0.0], [v], alpha, [1.0], family=O.FAMILY_NORMAL)
            qs = 1 + math.sqrt(-2 * math.log(alpha)) / v
            M = qs / (qs - 1) * math.log(alpha) - qs * v * v / 2
            assert abs(ap - math.exp(M)) <= 1e-12 * math.exp(M)
            assert abs(q - qs) <= 1e-8 * qs


def test_binomial_log_partition_by_enumeration():
    for n in (1, 10, 50, 100):
        for th in (-3.0, -0.5, 0.0, 1.7):
            x = np.arange(n + 1)
            A = special.logsumexp(th * x + np.log(special.comb(n, x)))
            assert abs(O.log_partition([th], [n]) - A) <= 1e-12 * max(1, abs(A))


def _logU_binomial(theta0, v, q, a, n):
    """log U by direct enumeration of psi(q) = log E_theta0[exp(q v T)] (Thm. tilt-bound).

    q may be an array; the result has its shape."""
    q = np.asarray(q, dtype=np.float64)
    tot = (1 - 1 / q) * math.log(a)
    x = np.arange(n + 1)
    for i in range(len(theta0)):
        p = 1 / (1 + math.exp(-theta0[i]))
        lp = np.log(stats.binom.pmf(x, n, p))
        psi_q = special.logsumexp(lp[None, :] + np.multiply.outer(q * v[i], x), axis=1)
        psi_1 = special.logsumexp(lp + v[i] * x)
        tot = tot + psi_q.reshape(q.shape) / q - psi_1
    return tot


@pytest.mark.parametrize("theta0,h,a,n", [
    ([-1 / 64], [1 / 64], 0.033272, 50),
    ([-1.5], [1 / 64], 5.62e-4, 50),
    ([0.3, 0.2], [1 / 128, 1 / 128], 0.0281, 100),
    ([-1.0, -1.9], [1 / 16, 1 / 16], 0.0007, 100),
    ([0.1, -0.2, 0.3, 0.0], [0.067, 0.067, 0.067, 0.067], 0.02, 40),
])
def test_binomial_tilt_bound_brute_force(theta0, h, a, n):
    d = len(theta0)
    b, q = O.tilt_bound(theta0, h, a, [n] * d)
    verts = [np.array([h[i] if (m >> i) & 1 else -h[i] for i in range(d)]) for m in range(1 << d)]
    # at q*, the bound equals the max over vertices of the enumerated log U
    if math.isfinite(q):
        lu = max(_logU_binomial(theta0, v, q, a, n) for v in verts)
        assert abs(math.exp(lu) - b) <= 1e-10 * b
    # no q on a fine log grid does better (Eq. optimized-tilt-bound-tile)
    qs = np.exp(np.linspace(0, 12, 4001))[1:]
    grid = np.max([_logU_binomial(theta0, v, qs, a, n) for v in verts], axis=0)
    gmin = math.exp(grid.min())
    assert b <= gmin * (1 + 1e-10)
    assert b >= gmin * (1 - 1e-3)


def test_tilt_bound_invariants():
    th, h, n = [-0.2], [1 / 64], [50]
    # increasing in a (Sec. 6.2), equal to 1 at a = 1, and at least a
    bs = [O.tilt_bound(th, h, a, n)[0] for a in (1e-4, 1e-3, 0.01, 0.03, 0.2)]
    assert all(y > x for x, y in zip(bs, bs[1:]))
    assert O.tilt_bound(th, h, 1.0, n)[0] == 1.0
    for a in (1e-4, 0.03):
        assert O.tilt_bound(th, h, a, n)[0] >= a
    # a zero-width tile gives back a
    b0, _ = O.tilt_bound(th, [1e-12], 0.03, n)
    assert abs(b0 - 0.03) < 1e-6


def test_vertex_max_dominates_interior():
    # Thm. 3: U is quasi-convex in v, so the vertex maximum bounds the whole box
    theta0, h, a, n = [0.2, -0.1], [0.05, 0.05], 0.02, 100
    b, q = O.tilt_bound(theta0, h, a, [n, n])
    for s0 in np.linspace(-1, 1, 9):
        for s1 in np.linspace(-1, 1, 9):
            v = [s0 * h[0], s1 * h[1]]
            assert math.exp(_logU_binomial(theta0, v, q, a, n)) <= b * (1 + 1e-12)


def test_alpha_prime_duality_and_brute_force():
    # U(theta0, v, q*, alpha') on the tile's vertices is at most alpha, and the
    # optimised bound from alpha' sits just below alpha (Eq. tile-calibration).
    for theta0, h, n in [([-1 / 64], [1 / 64], [50]), ([0.0, -0.3], [1 / 128, 1 / 128], [100, 100]),
                         ([0.1, 0.0, -0.2, 0.3], [0.067] * 4, [40] * 4)]:
        ap, q = O.alpha_prime(theta0, h, 0.025, n)
        assert 0 < ap < 0.025
        b, _ = O.tilt_bound(theta0, h, ap, n)
        assert b <= 0.025 * (1 + 1e-12)
        assert b >= 0.025 * (1 - 1e-6)
        d = len(theta0)
        verts = [np.array([h[i] if (m >> i) & 1 else -h[i] for i in range(d)]) for m in range(1 << d)]
        # brute-force max over q of min_v U^{-1}
        qq = np.exp(np.linspace(1e-4, 10, 3001))
        # psi(q)/q - psi(1) = log U(a) - (1 - 1/q) log a, at any a
        m = np.min([qq / (qq - 1) * (math.log(0.025) - (_logU_binomial(theta0, v, qq, 0.5, n[0])
                                                          - (1 - 1 / qq) * math.log(0.5)))
                    for v in verts], axis=0)
        best = m.max()
        assert ap >= math.exp(best) * (1 - 1e-10)
        assert ap <= math.exp(best) * (1 + 1e-3)


def test_order_statistic_index_pins():
    # k = floor((K + 1) alpha) at alpha = 0.025 (Eq. calibrated-threshold)
    for K, k in [(8192, 204), (16384, 409), (65536, 1638)]:
        assert math.floor((K + 1) * 0.025) == k
