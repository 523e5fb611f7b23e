"""GPU vs oracle parity of the randomised z-tests (Sec. 7: statistic (S, w),
threshold (lambda, c), lexicographic), through the C ABI.

Everything here is integer or table-valued, so bit for bit: per-tile pairs
(lambda_i, c_i), the lexicographic minimum, and reject counts / success sums
under a randomised threshold; the bounds from those counts within 1e-12.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2212_10042_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2212_10042_gb300 import binding
    binding.lib()
    return binding


def _np(t):
    return t.detach().cpu().numpy()


def _cases():
    rng = np.random.default_rng(21)
    one = W.one_arm_tiles(16, 2000, lo=-0.8, hi=0.0)
    rag = W.one_arm_tiles(24, 1, lo=-0.6, hi=0.0).with_K(rng.integers(1, 5001, size=24))
    two = W.two_arm_grid(16, 4096)
    return [("one_arm", W.ONE_ARM, one), ("one_arm_ragged", W.ONE_ARM, rag), ("two_arm", W.TWO_ARM, two)]


@pytest.mark.parametrize("name,design,tiles", _cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_calibrate_rand_matches_oracle(B, name, design, tiles):
    ctx = B.Context(design, K_max=int(tiles.K_max))
    dt = B.DeviceTiles(tiles)
    out = ctx.calibrate_rand(dt, 0.025)
    torch.cuda.synchronize()
    ctx.sync()
    ref = O.calibrate_rand(design, tiles, 0.025)
    assert np.allclose(_np(out["alpha_prime"]), ref["alpha_prime"], rtol=1e-12, atol=0)
    assert np.array_equal(_np(out["lambda_tile"]), ref["lambda_tile"])
    assert np.array_equal(_np(out["c_tile"]).view(np.uint32), ref["c_tile"])
    assert out["lam"] == ref["lam"] and out["c"] == ref["c"]


def test_validate_rand_matches_oracle_and_reduces_to_plain(B):
    design = W.TWO_ARM
    tiles = W.two_arm_grid(16, 4096)
    ctx = B.Context(design, K_max=4096)
    dt = B.DeviceTiles(tiles)
    cal = O.calibrate_rand(design, tiles, 0.025)
    lam, c = cal["lam"], cal["c"]
    # the calibrated pair (a table value with ties), a mid-word c, and c = 0
    for lam_i, c_i in [(lam, c), (lam, 1 << 31), (float(cal["lambda_tile"][5]), int(cal["c_tile"][5])), (lam, 0)]:
        out = ctx.validate_rand(dt, lam_i, c_i, 0.01)
        torch.cuda.synchronize()
        ctx.sync()
        ref = O.simulate_rand(design, tiles, lam_i, c_i)
        assert np.array_equal(_np(out["R"]), ref["R"])
        assert np.array_equal(_np(out["Xrej"]), ref["Xrej"])
        bnd = O.validate_bounds(design, tiles, ref["R"], 0.01)
        assert np.allclose(_np(out["bound"]), bnd["bound"], rtol=1e-12, atol=0)
        if c_i == 0:
            plain = ctx.validate(dt, lam_i, 0.01)
            assert torch.equal(out["R"], plain["R"]) and torch.equal(out["Xrej"], plain["Xrej"])


def test_calibrated_pairs_reject_k_minus_one(B):
    design = W.ONE_ARM
    tiles = W.one_arm_tiles(12, 3000, lo=-0.6, hi=0.0)
    ctx = B.Context(design, K_max=3000)
    dt = B.DeviceTiles(tiles)
    out = ctx.calibrate_rand(dt, 0.025)
    lt, ct = _np(out["lambda_tile"]), _np(out["c_tile"]).view(np.uint32)
    kk = O.calibrate_rand(design, tiles, 0.025)["k"]
    for i in range(tiles.n_tiles):
        sub = B.DeviceTiles(tiles.subset([i]))
        r = ctx.validate_rand(sub, float(lt[i]), int(ct[i]), 0.01)["R"]
        torch.cuda.synchronize()
        assert int(r.item()) == int(kk[i]) - 1


def test_bayes_design_is_refused(B):
    ctx = B.Context(W.BAYES4, K_max=64)
    dt = B.DeviceTiles(W.four_arm_grid(2, 64))
    with pytest.raises(B.CseError):
        ctx.calibrate_rand(dt, 0.025)


@pytest.mark.parametrize("name,design,tiles", _cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_rand_cells_path_equals_plain_path(B, name, design, tiles):
    """The chosen form (cell-histogram pass + tie pass) and the plain per-sim
    kernel give identical pairs, counts, success sums and scores, including
    lambda = 0, where the two-arm statistic ties along the whole diagonal
    x0 = x1 (more tie cells than the tie pass keeps in registers), and
    calibration at alpha = 0.5 (order statistics near that diagonal)."""
    ctx = B.Context(design, K_max=int(tiles.K_max))
    dt = B.DeviceTiles(tiles)

    def run():
        out = {}
        for alpha in (0.025, 0.5):
            r = ctx.calibrate_rand(dt, alpha)
            torch.cuda.synchronize()
            out[("cal", alpha)] = (_np(r["lambda_tile"]).copy(), _np(r["c_tile"]).copy(), r["lam"], r["c"])
        lam = out[("cal", 0.025)][2]
        c = out[("cal", 0.025)][3]
        for lam_i, c_i in [(lam, c), (lam, 1 << 31), (0.0, 1 << 31), (0.0, 0), (-1.5, 12345)]:
            v = ctx.validate_rand(dt, lam_i, c_i, 0.01)
            torch.cuda.synchronize()
            out[("val", lam_i, c_i)] = (_np(v["R"]).copy(), _np(v["Xrej"]).copy(), _np(v["score"]).copy())
        ctx.sync()
        return out

    chosen = run()
    ctx.set_option(B.OPT_PLAIN, 1)
    plain = run()
    assert chosen.keys() == plain.keys()
    for key in chosen:
        for a, b in zip(chosen[key], plain[key]):
            assert np.array_equal(np.asarray(a), np.asarray(b)), key
    # the diagonal case against the oracle as well
    ref = O.simulate_rand(design, tiles, 0.0, 1 << 31)
    assert np.array_equal(chosen[("val", 0.0, 1 << 31)][0], ref["R"])
    cal = O.calibrate_rand(design, tiles, 0.5)
    assert np.array_equal(chosen[("cal", 0.5)][0], cal["lambda_tile"])
    assert np.array_equal(chosen[("cal", 0.5)][1].view(np.uint32), cal["c_tile"])


def test_rand_large_tie_groups(B):
    """One-arm design at K = 65,536: at alpha = 0.5 the selected rank's cell holds
    thousands of sims, more than the tie pass keeps in shared memory, so its
    words spill to the global buffer and go through the radix select.  Chosen,
    plain and oracle agree bit for bit."""
    design = W.ONE_ARM
    tiles = W.one_arm_tiles(4, 65536, lo=-0.4, hi=0.0)
    ctx = B.Context(design, K_max=65536)
    dt = B.DeviceTiles(tiles)
    got = {}
    for plain in (0, 1):
        ctx.set_option(B.OPT_PLAIN, plain)
        for alpha in (0.5, 0.025):
            r = ctx.calibrate_rand(dt, alpha)
            torch.cuda.synchronize()
            got[(plain, alpha)] = (_np(r["lambda_tile"]).copy(), _np(r["c_tile"]).view(np.uint32).copy())
    ctx.sync()
    for alpha in (0.5, 0.025):
        ref = O.calibrate_rand(design, tiles, alpha)
        for plain in (0, 1):
            assert np.array_equal(got[(plain, alpha)][0], ref["lambda_tile"]), (plain, alpha)
            assert np.array_equal(got[(plain, alpha)][1], ref["c_tile"]), (plain, alpha)
    # the groups really exceed the shared-memory part: at alpha = 0.5 the sims
    # tying the selected statistic number over 2,048 (one-arm cells are ranks)
    S = O.simulate(design, tiles, 0.0, want_S=True)["S"]
    lam_half = got[(0, 0.5)][0]
    assert max(int(np.sum(S[i] == lam_half[i])) for i in range(tiles.n_tiles)) > 2048
