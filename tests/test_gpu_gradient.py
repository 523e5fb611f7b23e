"""The differentiable Type I Error (TypeIError autograd function) on the GPU.

Its backward is the score-function adjoint (Ex. exp-fam): d f/d theta =
E[F (T - grad A)].  Checked against the exact derivative of the one-arm test,
50 C(49,31) p^32 (1-p)^19, and against common-random-number central finite
differences of the same Monte Carlo estimate.  With CRN and a rejection region
monotone in theta, the two FD arms differ only on the trials that reject at
theta+h but not at theta-h, so Var(FD) <= (f(theta+h) - f(theta-h)) / (4 h^2 K)
exactly, and each estimator is tested within 4.5 standard deviations.
"""
import math

import numpy as np
import pytest
import torch
from scipy import stats

from oracle import oracle as O
from paper_2212_10042_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2212_10042_gb300 import binding
    binding.lib()
    return binding


def _exact(theta):
    p = O.threshold(theta) / 2.0 ** 32
    f = stats.binom.sf(31, 50, p)
    df = 50 * math.comb(49, 31) * p ** 32 * (1 - p) ** 19
    x = np.arange(51)
    pm = stats.binom.pmf(x, 50, p)
    g = (x >= 32) * (x - 50 * p)
    var_score = (g ** 2 * pm).sum() - df ** 2
    return f, df, var_score


@pytest.mark.parametrize("theta", [-0.3, 0.0])
def test_score_gradient_exact_and_crn_fd(B, theta):
    K, h = 1 << 17, 0.05
    ctx = B.Context(W.ONE_ARM, seed=2024, K_max=K)
    th = torch.tensor([[theta]], dtype=torch.float64, device="cuda", requires_grad=True)
    f = B.TypeIError.apply(th, ctx, 1, K, -1.96)
    f.sum().backward()
    grad = th.grad.item()
    _, df, var_score = _exact(theta)
    assert abs(grad - df) <= 4.5 * math.sqrt(var_score / K)
    # common-random-number central differences of the same estimator
    with torch.no_grad():
        pts = torch.tensor([[theta + h], [theta - h]], dtype=torch.float64, device="cuda")
        fp, fm = B.TypeIError.apply(pts, ctx, 1, K, -1.96).tolist()
    fd = (fp - fm) / (2 * h)
    f_plus, _, _ = _exact(theta + h)
    f_minus, _, _ = _exact(theta - h)
    fd_exact = (f_plus - f_minus) / (2 * h)            # the FD estimator's mean
    sd_fd = math.sqrt(max(f_plus - f_minus, 1e-300) / (4 * h * h * K))
    assert abs(fd - fd_exact) <= 4.5 * sd_fd + 1e-12
    # the FD's own bias is O(h^2); both estimate the same derivative
    assert abs(fd_exact - df) <= 0.05 * df
    assert abs(grad - fd) <= 4.5 * (math.sqrt(var_score / K) + sd_fd) + abs(fd_exact - df)
