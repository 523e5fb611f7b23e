"""GPU vs oracle for the four-arm Bayesian selection design, through the C ABI.

The GPU evaluates the posterior in FP32, the oracle in FP64, so a decision can
flip when a posterior probability lies within FP32 rounding of a threshold:
flips are counted and bounded, every other quantity is compared exactly or to
its stated tolerance:
  - success counts (via the tabulated and the direct posterior modes, which
    must agree bit for bit with each other),
  - |S_gpu - S_oracle| <= 2e-5 on trials without a flipped drop decision,
  - lambda_tile equals the exact k-th order statistic of the GPU's own S,
  - alpha' and k = floor((K+1) alpha') against the oracle (1e-12 / exact),
  - FP64 bounds from the GPU's reject counts against the oracle's (1e-12).
"""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2212_10042_gb300 import workloads as W

pytestmark = pytest.mark.gpu

S_TOL = 2e-5          # |S_gpu - S_oracle| for an FP32 posterior (S in [0, 1])
FLIP_RATE = 1e-3      # bound on trials whose FP32 decisions differ from FP64


@pytest.fixture(scope="module")
def B():
    from paper_2212_10042_gb300 import binding
    binding.lib()
    return binding


def _np(t):
    return t.detach().cpu().numpy()


def _sample_tiles(tiles, n, seed):
    rng = np.random.default_rng(seed)
    return tiles.subset(np.sort(rng.choice(tiles.n_tiles, n, replace=False)))


def _compare_stats(S_gpu, off, ref_S, K):
    flips = 0
    n = 0
    for i, Sr in enumerate(ref_S):
        Sg = S_gpu[off[i]: off[i] + K[i]].astype(np.float64)
        fin = np.isfinite(Sr) & np.isfinite(Sg)
        d = np.abs(np.where(fin, Sg, 0.0) - np.where(fin, Sr, 0.0))   # both +inf: no difference
        mism = (np.isfinite(Sr) != np.isfinite(Sg)) | (fin & (d > S_TOL))
        flips += int(mism.sum())
        n += len(Sr)
    return flips, n


def test_bayes4_small_against_oracle(B):
    design = W.BAYES4
    tiles = _sample_tiles(W.four_arm_grid(16, 4096), 24, 1)
    ctx = B.Context(design, K_max=4096)
    dt = B.DeviceTiles(tiles)
    lam = 0.06
    out = ctx.step(dt, lam, 0.01, 0.025)
    S, off = ctx.statistics(dt)
    torch.cuda.synchronize()
    ctx.sync()
    S, off = _np(S), _np(off)
    ref = O.simulate(design, tiles, lam, want_S=True)
    flips, n = _compare_stats(S, off, ref["S"], tiles.K)
    assert flips <= FLIP_RATE * n, (flips, n)
    # reject counts: internally consistent with the GPU's statistics, and within
    # the flips of the oracle's
    R = _np(out["R"])
    for i in range(tiles.n_tiles):
        Sg = S[off[i]: off[i] + tiles.K[i]].astype(np.float64)
        assert R[i] == int((Sg < lam).sum())
    assert np.abs(R - ref["R"]).sum() <= flips
    # selection is exact on the GPU's own statistics
    ap = _np(out["alpha_prime"])
    lt = _np(out["lambda_tile"])
    cal = O.calibrate(design, tiles, 0.025)
    assert np.allclose(ap, cal["alpha_prime"], rtol=1e-12, atol=0)
    k = np.minimum(np.floor((tiles.K + 1.0) * ap).astype(np.int64), tiles.K)
    assert np.array_equal(k, cal["k"])
    for i in range(tiles.n_tiles):
        Sg = np.sort(S[off[i]: off[i] + tiles.K[i]])
        want = -math.inf if k[i] < 1 else float(Sg[k[i] - 1])
        assert lt[i] == want
    fin = np.isfinite(cal["lambda_tile"])
    assert np.all(np.abs(lt[fin] - cal["lambda_tile"][fin]) <= S_TOL)
    # FP64 bound pass from the GPU's counts against the oracle's bound pass
    vb = O.validate_bounds(design, tiles, R, 0.01)
    assert np.allclose(_np(out["bound"]), vb["bound"], rtol=1e-12, atol=0)
    assert np.allclose(_np(out["u0"]), vb["u0"], rtol=1e-12, atol=0)


def test_bayes4_tables_match_direct_posterior(B):
    design = W.BAYES4
    tiles = _sample_tiles(W.four_arm_grid(16, 2048), 40, 2)
    ctx = B.Context(design, K_max=2048)
    dt = B.DeviceTiles(tiles)
    a = ctx.step(dt, 0.06, 0.01, 0.025)
    Sa, _ = ctx.statistics(dt)
    a = {k: v.clone() for k, v in a.items()}
    ctx.set_option(B.OPT_BAYES_DIRECT, 1)
    b = ctx.step(dt, 0.06, 0.01, 0.025)
    Sb, _ = ctx.statistics(dt)
    torch.cuda.synchronize()
    assert torch.equal(Sa, Sb)
    for key in ("R", "Xrej", "lambda_tile"):
        assert torch.equal(a[key], b[key]), key


def test_bayes4_ragged_and_masks(B):
    # one-hypothesis masks, K not a multiple of the block, K = 1
    design = W.BAYES4
    base = _sample_tiles(W.four_arm_grid(16, 1), 16, 3)
    rng = np.random.default_rng(4)
    tiles = base.with_K(rng.integers(1, 1500, size=base.n_tiles))
    tiles.K[0] = 1
    tiles.null_mask[:] = np.array([1, 2, 4, 3, 5, 6, 7, 1] * 2, dtype=np.uint32)
    ctx = B.Context(design, K_max=1500)
    dt = B.DeviceTiles(tiles)
    out = ctx.step(dt, 0.1, 0.05, 0.05)
    S, off = ctx.statistics(dt)
    torch.cuda.synchronize()
    ctx.sync()
    ref = O.simulate(design, tiles, 0.1, want_S=True)
    flips, n = _compare_stats(_np(S), _np(off), ref["S"], tiles.K)
    assert flips <= max(2, FLIP_RATE * n)
    assert np.abs(_np(out["R"]) - ref["R"]).sum() <= flips


@pytest.mark.parametrize("cfg,n_sample", [("c4", 6), ("c5", 3)])
def test_bayes4_full_size_sampled(B, cfg, n_sample):
    """Full-size platten in the benchmark's launch configuration; sampled tiles
    recomputed by the oracle."""
    design, tiles = W.CONFIGS[cfg]()
    ctx = B.Context(design, K_max=tiles.K_max)
    dt = B.DeviceTiles(tiles)
    out = ctx.step(dt, 0.06, 0.01, 0.025)
    torch.cuda.synchronize()
    ctx.sync()
    R, lt, ap = _np(out["R"]), _np(out["lambda_tile"]), _np(out["alpha_prime"])
    rng = np.random.default_rng(9)
    rows = np.unique(np.concatenate([[int(np.argmin(lt)), int(np.argmax(R))],
                                     rng.choice(tiles.n_tiles, n_sample, replace=False)]))
    sub = tiles.subset(rows)
    ref = O.simulate(design, sub, 0.06)
    tol = max(3, int(1e-3 * sub.K.max()))
    assert np.all(np.abs(R[rows] - ref["R"]) <= tol)
    cal = O.calibrate(design, sub, 0.025)
    assert np.allclose(ap[rows], cal["alpha_prime"], rtol=1e-12, atol=0)
    fin = np.isfinite(cal["lambda_tile"])
    assert np.all(np.abs(lt[rows][fin] - cal["lambda_tile"][fin]) <= S_TOL)
    vb = O.validate_bounds(design, sub, R[rows], 0.01)
    assert np.allclose(_np(out["bound"])[rows], vb["bound"], rtol=1e-12, atol=0)
    assert out["lam"].item() == lt.min()



def test_bayes4_byte_form_tables_design(B):
    """A design whose final-look codes do not fit seven bits (looks 20/40/70:
    133 codes) runs the byte-form tabulated kernel (256 threads) instead of the
    packed one (512 threads, the 10/20/40 design).  Both forms read the same
    tables: the statistics and the step's outputs agree bit for bit with the
    direct per-trial posterior, and with the oracle within the FP32 flips."""
    design = W.Design("bayes4_looks_20_40_70", "bayes4", 4, (20, 40, 70))
    tiles = _sample_tiles(W.four_arm_grid(16, 512), 8, 5)
    ctx = B.Context(design, K_max=512)
    dt = B.DeviceTiles(tiles)
    assert ctx.autotune(dt, 0.06, 0.025)[0] == 256
    a = {k: v.clone() for k, v in ctx.step(dt, 0.06, 0.01, 0.025).items()}
    Sa, off = ctx.statistics(dt)
    Sa = Sa.clone()
    ctx.set_option(B.OPT_BAYES_DIRECT, 1)
    b = ctx.step(dt, 0.06, 0.01, 0.025)
    Sb, _ = ctx.statistics(dt)
    torch.cuda.synchronize()
    ctx.sync()
    assert torch.equal(Sa, Sb)
    for key in ("R", "Xrej", "lambda_tile"):
        assert torch.equal(a[key], b[key]), key
    ref = O.simulate(design, tiles, 0.06, want_S=True)
    flips, n = _compare_stats(_np(Sa), _np(off), ref["S"], tiles.K)
    assert flips <= max(2, FLIP_RATE * n), (flips, n)
    # the benchmark design runs the packed form
    c2 = B.Context(W.BAYES4, K_max=512)
    assert c2.autotune(dt, 0.06, 0.025)[0] == 512


def test_bayes4_non_selecting_kernel_matches_the_step(B):
    """The validation entry points run the non-selecting form of the four-arm
    kernel and mark the Clopper-Pearson keys with k_cp_mark; the step runs the
    selecting form, which inserts the keys itself.  Same trials, so R, Xrej
    and the score agree bit for bit, and so do the bounds computed from them."""
    design = W.BAYES4
    tiles = _sample_tiles(W.four_arm_grid(16, 2048), 40, 6)
    ctx = B.Context(design, K_max=2048)
    dt = B.DeviceTiles(tiles)
    a = {k: v.clone() for k, v in ctx.step(dt, 0.06, 0.01, 0.025).items()}
    R, X, G = ctx.simulate_tiles(dt, 0.06)
    v = ctx.validate(dt, 0.06, 0.01)
    band = ctx.validate_band(dt, 0.06, 0.01)
    torch.cuda.synchronize()
    ctx.sync()
    for r in (R, v["R"], band["R"]):
        assert torch.equal(r, a["R"])
    for x in (X, v["Xrej"]):
        assert torch.equal(x, a["Xrej"])
    assert torch.equal(G, a["score"])
    assert torch.equal(v["u0"], a["u0"])
    assert np.allclose(_np(v["bound"]), _np(a["bound"]), rtol=1e-14, atol=0)
    ref = O.simulate(design, tiles, 0.06)
    assert np.abs(_np(R) - ref["R"]).sum() <= max(2, int(FLIP_RATE * tiles.K.sum()))
