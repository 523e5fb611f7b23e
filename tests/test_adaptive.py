"""The adaptive calibration loop (paper_2212_10042_gb300/adaptive.py): its tile
geometry, its rule against a synthetic calibrator, and a full loop driven by
the oracle's calibration on a one-arm platten."""
import numpy as np

from oracle import oracle as O
from paper_2212_10042_gb300 import adaptive as A
from paper_2212_10042_gb300 import workloads as W


def _orc(design, alpha):
    def f(t):
        r = O.calibrate(design, t, alpha)
        return r["alpha_prime"], r["lambda_tile"], r["lam"]
    return f


def test_children_tile_the_parent_and_keep_the_null_set():
    # tile 0: [0, 0.5]^2 crosses theta1 = theta0; tile 1: entirely below it
    t = W.from_centers([[0.25, 0.25], [0.5, -0.5]], [[0.25, 0.25], [0.125, 0.125]], [1, 1], [100, 200])
    ch = A.split(t, [0, 1], one_arm=False)
    c, h = ch.centers, ch.halfwidth
    assert ch.n_tiles == 7
    # every kept child meets theta1 <= theta0
    assert np.all(W.null_mask_of_boxes(c, h, one_arm=False) != 0)
    # tile 0 loses the child strictly above the diagonal, (0.125, 0.375)
    top = c[np.isclose(h[:, 0], 0.125)]
    assert len(top) == 3 and not any(np.allclose(x, [0.125, 0.375]) for x in top)
    assert np.all(ch.K[np.isclose(h[:, 0], 0.125)] == 100)
    # the children of tile 1 tile its box exactly and keep its K
    kids = c[np.isclose(h[:, 0], 0.0625)]
    assert len(kids) == 4
    assert np.allclose((kids - 0.0625).min(0), [0.375, -0.625]) and np.allclose((kids + 0.0625).max(0), [0.625, -0.375])
    assert set(np.round(kids[:, 0], 6)) == {0.4375, 0.5625} and set(np.round(kids[:, 1], 6)) == {-0.5625, -0.4375}
    assert np.all(ch.K[np.isclose(h[:, 0], 0.0625)] == 200)


def test_rule_against_a_synthetic_calibrator():
    cfg = A.RefineConfig(alpha=0.025, crit_frac=0.25, slack_tol=0.1, min_halfwidth=1 / 64, K_cap=4096)
    t = W.one_arm_tiles(8, 1024, lo=-1.0, hi=0.0)           # h = 1/16
    lam = np.array([-2.0, -1.9, -1.8, -1.7, -1.6, -1.5, -1.4, -1.3])
    ap = np.full(8, 0.025 * 0.85)                             # slack 0.15 > 0.1
    ap[1] = 0.025 * 0.95                                      # slack 0.05: double K instead
    new, n_split, n_double = A.refine(t, ap, lam, cfg, one_arm=True)
    assert (n_split, n_double) == (1, 1)                      # lowest 25%: tiles 0 and 1
    assert new.n_tiles == 9 and sorted(new.K.tolist()).count(2048) == 1
    # -inf (k = 0) doubles K first, whatever its slack
    lam2 = lam.copy()
    lam2[3] = -np.inf
    _, n_split, n_double = A.refine(t, ap, lam2, cfg, one_arm=True)
    assert n_double >= 1
    # at the cap and at the smallest half-width nothing changes
    tc = t.with_K(4096)
    tc.halfwidth[:] = 1 / 64
    _, n_split, n_double = A.refine(tc, ap, lam, cfg, one_arm=True)
    assert (n_split, n_double) == (0, 0)


def test_oracle_driven_loop_converges_and_raises_lambda():
    t0 = W.one_arm_tiles(8, 512, lo=-1.0, hi=0.0)
    cfg = A.RefineConfig(alpha=0.025, max_iter=8, crit_frac=0.25, slack_tol=0.05, min_halfwidth=1 / 128,
                         K_cap=4096)
    res = A.run(t0, _orc(W.ONE_ARM, 0.025), cfg, one_arm=True)
    tr = res["trace"]
    assert tr[0]["split"] > 0
    final = res["tiles"]
    crit = A.critical(res["lambda_tile"], cfg)
    slack = (cfg.alpha - res["alpha_prime"]) / cfg.alpha
    # on convergence every critical tile is tight, at the smallest size, or at the K cap
    if res["converged"]:
        assert np.all(~crit | (slack <= cfg.slack_tol) | (final.halfwidth[:, 0] / 2 < cfg.min_halfwidth)
                      | (final.K >= cfg.K_cap))
    # the platten still covers [-1, 0] exactly: half-widths sum to the length
    assert abs(2 * final.halfwidth[:, 0].sum() - 1.0) < 1e-12
    # every tile's alpha' <= alpha, and lambda* never below the first round's
    assert np.all(res["alpha_prime"] <= cfg.alpha)
    assert res["lam"] >= tr[0]["lam"]
