"""The adaptive calibration loop on the GPU path against the same loop driven by
the oracle's calibration: every round's platten and lambda* are identical
(lambda_i are elements of the FP32 statistic table, so bit for bit), and the
final alpha'_i agree within 1e-12 relative."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2212_10042_gb300 import adaptive as A
from paper_2212_10042_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _orc(design, alpha):
    def f(t):
        r = O.calibrate(design, t, alpha)
        return r["alpha_prime"], r["lambda_tile"], r["lam"]
    return f


def _same_platten(a, b):
    assert a.n_tiles == b.n_tiles
    oa = np.lexsort(np.c_[a.centers, a.halfwidth].T)
    ob = np.lexsort(np.c_[b.centers, b.halfwidth].T)
    assert np.array_equal(a.centers[oa], b.centers[ob])
    assert np.array_equal(a.halfwidth[oa], b.halfwidth[ob])
    assert np.array_equal(a.K[oa], b.K[ob]) and np.array_equal(a.null_mask[oa], b.null_mask[ob])


@pytest.mark.parametrize("case", ["one_arm", "two_arm"])
def test_adaptive_loop_matches_oracle_loop(case):
    if case == "one_arm":
        design, t0, one = W.ONE_ARM, W.one_arm_tiles(8, 512, lo=-1.0, hi=0.0), True
        cfg = A.RefineConfig(alpha=0.025, max_iter=6, crit_frac=0.25, slack_tol=0.05,
                             min_halfwidth=1 / 128, K_cap=4096)
    else:
        design, t0, one = W.TWO_ARM, W.two_arm_grid(8, 1024), False
        cfg = A.RefineConfig(alpha=0.025, max_iter=4, crit_frac=0.1, slack_tol=0.05,
                             min_halfwidth=1 / 64, K_cap=8192)
    gpu = A.run(t0, A.GpuCalibrator(design, cfg.alpha, cfg.K_cap), cfg, one_arm=one)
    orc = A.run(t0, _orc(design, cfg.alpha), cfg, one_arm=one)
    assert gpu["trace"] == orc["trace"]
    assert gpu["converged"] == orc["converged"]
    _same_platten(gpu["tiles"], orc["tiles"])
    assert gpu["lam"] == orc["lam"]
    # the final calibration, tile for tile (both loops list tiles in the same order)
    assert np.array_equal(gpu["lambda_tile"], orc["lambda_tile"])
    assert np.allclose(gpu["alpha_prime"], orc["alpha_prime"], rtol=1e-12, atol=0)
    first = gpu["trace"][0]
    assert len(gpu["trace"]) >= 2 and first["split"] + first["doubled"] > 0
