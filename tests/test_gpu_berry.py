"""GPU vs oracle for the basket trial of Sec. 10.1 (four arms, n = 35, one
analysis, reject arm i when P(theta_i > t_i | x) > 85%), through the C ABI.

The GPU tabulates the posterior in FP32, the oracle evaluates it in FP64 per
trial, so a decision can flip when 1 - P_i lies within FP32 rounding of lambda:
flips are counted and bounded; everything else is compared exactly or to its
stated tolerance:
  - |S_gpu - S_oracle| <= 2e-5 per trial (more counts as a flip),
  - R equals the count of the GPU's own S below lambda, and the oracle's R
    within the flips,
  - lambda_tile is exactly the k-th order statistic of the GPU's own S,
  - alpha' and k = floor((K+1) alpha') against the oracle (1e-12 / exact),
  - the table and the direct per-trial posterior agree bit for bit,
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
FLIP_RATE = 1e-3      # bound on trials whose FP32 statistic strays beyond S_TOL
LAM = W.BERRY_LAMBDA


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
    flips = n = 0
    worst = 0.0
    for i, Sr in enumerate(ref_S):
        Sg = S_gpu[off[i]: off[i] + K[i]].astype(np.float64)
        fin = np.isfinite(Sr) & np.isfinite(Sg)
        d = np.abs(Sg - Sr)
        mism = (np.isfinite(Sr) != np.isfinite(Sg)) | (fin & (d > S_TOL))
        flips += int(mism.sum())
        n += len(Sr)
        if fin.any():
            worst = max(worst, float(d[fin].max()))
    return flips, n, worst


def test_berry_small_against_oracle(B):
    design = W.BERRY4
    tiles = _sample_tiles(W.berry_grid(16, 4096), 24, 1)
    ctx = B.Context(design, K_max=4096)
    dt = B.DeviceTiles(tiles)
    out = ctx.step(dt, LAM, 0.01, 0.025)
    S, off = ctx.statistics(dt)
    torch.cuda.synchronize()
    ctx.sync()
    S, off = _np(S), _np(off)
    ref = O.simulate(design, tiles, LAM, want_S=True)
    flips, n, worst = _compare_stats(S, off, ref["S"], tiles.K)
    assert flips <= FLIP_RATE * n, (flips, n, worst)
    R = _np(out["R"])
    assert R.sum() > 0      # the sample rejects: the comparison is not vacuous
    for i in range(tiles.n_tiles):
        Sg = S[off[i]: off[i] + tiles.K[i]].astype(np.float64)
        assert R[i] == int((Sg < LAM).sum())
    assert np.abs(R - ref["R"]).sum() <= flips
    # success sums of the rejected trials: exact where no trial flipped
    same = R == ref["R"]
    assert np.array_equal(_np(out["Xrej"])[same], ref["Xrej"][same])
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
    vb = O.validate_bounds(design, tiles, R, 0.01)
    assert np.allclose(_np(out["bound"]), vb["bound"], rtol=1e-12, atol=0)
    assert np.allclose(_np(out["u0"]), vb["u0"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("K,n", [(2048, 40), (16384, 12)])
def test_berry_table_matches_direct_posterior(B, K, n):
    """Table path (with the shared-memory statistic box when K >= its states,
    as at K = 2^14) and direct per-trial posterior agree bit for bit."""
    design = W.BERRY4
    tiles = _sample_tiles(W.berry_grid(16, K), n, 2)
    ctx = B.Context(design, K_max=K)
    dt = B.DeviceTiles(tiles)
    a = ctx.step(dt, LAM, 0.01, 0.025)
    Sa, _ = ctx.statistics(dt)
    a = {k: v.clone() for k, v in a.items()}
    ctx.set_option(B.OPT_BAYES_DIRECT, 1)
    b = ctx.step(dt, LAM, 0.01, 0.025)
    Sb, _ = ctx.statistics(dt)
    torch.cuda.synchronize()
    assert torch.equal(Sa, Sb)
    for key in ("R", "Xrej", "score", "lambda_tile"):
        assert torch.equal(a[key], b[key]), key


def test_berry_validate_ragged_and_masks(B):
    # every mask 1..15, K = 1, K not a multiple of the 8 sims a thread takes per step
    design = W.BERRY4
    base = _sample_tiles(W.berry_grid(16, 1), 30, 3)
    rng = np.random.default_rng(4)
    tiles = base.with_K(rng.integers(1, 1500, size=base.n_tiles))
    tiles.K[0] = 1
    tiles.K[1] = 8
    tiles.K[2] = 9
    tiles.null_mask[:] = (np.arange(base.n_tiles) % 15 + 1).astype(np.uint32)
    ctx = B.Context(design, K_max=1500)
    dt = B.DeviceTiles(tiles)
    out = ctx.validate(dt, 0.3, 0.05)
    S, off = ctx.statistics(dt)
    torch.cuda.synchronize()
    ctx.sync()
    ref = O.simulate(design, tiles, 0.3, want_S=True)
    flips, n, worst = _compare_stats(_np(S), _np(off), ref["S"], tiles.K)
    assert flips <= max(2, FLIP_RATE * n), (flips, worst)
    assert np.abs(_np(out["R"]) - ref["R"]).sum() <= flips
    vb = O.validate_bounds(design, tiles, _np(out["R"]), 0.05)
    assert np.allclose(_np(out["bound"]), vb["bound"], rtol=1e-12, atol=0)


def test_berry_full_size_sampled(B):
    """The benchmark's platten (16^4 grid over [-3.5, 1]^4, K = 2^14) in its launch
    configuration; sampled tiles recomputed by the oracle."""
    design, tiles = W.CONFIGS["berry"]()
    ctx = B.Context(design, K_max=tiles.K_max)
    dt = B.DeviceTiles(tiles)
    out = ctx.step(dt, LAM, 0.01, 0.025)
    torch.cuda.synchronize()
    ctx.sync()
    R, lt, ap = _np(out["R"]), _np(out["lambda_tile"]), _np(out["alpha_prime"])
    rng = np.random.default_rng(9)
    rows = np.unique(np.concatenate([[int(np.argmin(lt)), int(np.argmax(R))],
                                     rng.choice(tiles.n_tiles, 6, replace=False)]))
    sub = tiles.subset(rows)
    ref = O.simulate(design, sub, LAM)
    tol = max(3, int(1e-3 * sub.K.max()))
    assert np.all(np.abs(R[rows] - ref["R"]) <= tol)
    cal = O.calibrate(design, sub, 0.025)
    assert np.allclose(ap[rows], cal["alpha_prime"], rtol=1e-12, atol=0)
    fin = np.isfinite(cal["lambda_tile"])
    assert np.all(np.abs(lt[rows][fin] - cal["lambda_tile"][fin]) <= S_TOL)
    vb = O.validate_bounds(design, sub, R[rows], 0.01)
    assert np.allclose(_np(out["bound"])[rows], vb["bound"], rtol=1e-12, atol=0)
    assert out["lam"].item() == lt.min()


def test_berry_refuses_bad_designs(B):
    with pytest.raises(B.CseError):
        B.Context(W.Design("berry4_n70", "berry4", 4, (70,), arm_null=W.BERRY4.arm_null), K_max=64)
    with pytest.raises(B.CseError):
        B.Context(W.Design("berry4_2looks", "berry4", 4, (10, 35), arm_null=W.BERRY4.arm_null), K_max=64)
    ctx = B.Context(W.BERRY4, K_max=64)
    dt = B.DeviceTiles(W.berry_grid(2, 64))
    with pytest.raises(B.CseError):
        ctx.calibrate_rand(dt, 0.025)
