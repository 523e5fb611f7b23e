"""GPU vs oracle parity of the lower validation bound and the two-sided band
(Rem. extension-lower), through the C ABI.

Reject counts bit for bit; the lower Clopper-Pearson bound l0 within 1e-12
relative.  The lower tile bound is lower = 1 - U with U the tile Tilt-Bound at
a = 1 - l0, so it is held to the upper bound's bar on U, 1e-12 relative:
|d lower| <= 1e-12 (1 - lower).  (A relative bar on lower itself is not
attainable: the q-search fixes log U to ~1e-14 absolute, which for a lower
bound of 1e-6 is 1e-8 relative; measured 1.3e-14 on the GPU.)  q* where the
inner bound is well conditioned (U <= 0.999, i.e. lower >= 0.001).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2212_10042_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def B():
    from paper_2212_10042_gb300 import binding
    binding.lib()
    return binding


def _np(t):
    return t.detach().cpu().numpy()


def _check_lower(out, ref):
    assert np.allclose(_np(out["l0"]), ref["l0"], rtol=RTOL, atol=0)
    lo = _np(out["lower"])
    assert np.all(lo >= 0.0)
    assert np.all(np.abs(lo - ref["lower"]) <= RTOL * (1.0 - ref["lower"]) + 1e-300)
    q, qr = _np(out["qstar"]), ref["qstar"]
    assert np.array_equal(np.isinf(q), np.isinf(qr))
    sharp = ~np.isinf(qr) & (ref["lower"] >= 1e-3)
    assert np.all(q[~np.isinf(qr)] >= 1.0)
    assert np.all(np.abs(q[sharp] - qr[sharp]) <= 1e-6 * np.abs(qr[sharp]))


def test_one_arm_full_config_lower(B):
    design, tiles = W.CONFIGS["c1"]()
    ctx = B.Context(design, K_max=tiles.K_max)
    out = ctx.validate_lower(B.DeviceTiles(tiles), -1.96, 0.01)
    torch.cuda.synchronize()
    ctx.sync()
    ref = O.simulate(design, tiles, -1.96)
    assert np.array_equal(_np(out["R"]), ref["R"])
    _check_lower(out, O.validate_lower(design, tiles, ref["R"], 0.01))


def test_lower_across_R_and_K(B):
    """R from 0 to K and ragged K up to 2^16 (R = 0: l0 = 0 without a solve;
    R = K: l0 = delta^(1/K)); more distinct (K, R - 1) keys than the warp slots."""
    design = W.ONE_ARM
    rng = np.random.default_rng(12)
    n = 1500
    c = np.linspace(-0.5, 2.0, n)[:, None]
    h = np.full_like(c, 1.25 / n)
    K = rng.integers(1, 4097, size=n).astype(np.int32)
    big = rng.choice(n, size=24, replace=False)
    K[big] = rng.integers(4097, (1 << 16) + 1, size=24)
    K[:3] = [1, 2, 1 << 16]
    tiles = W.from_centers(c, h, np.ones(n, dtype=np.uint32), K)
    ctx = B.Context(design, K_max=1 << 16)
    out = ctx.validate_lower(B.DeviceTiles(tiles), -1.96, 0.05)
    torch.cuda.synchronize()
    ctx.sync()
    ref = O.simulate(design, tiles, -1.96)
    R = ref["R"]
    assert np.array_equal(_np(out["R"]), R)
    assert (R == 0).any() and (R == tiles.K).any()
    _check_lower(out, O.validate_lower(design, tiles, R, 0.05))


@pytest.mark.parametrize("cells,K", [(16, 4096), (32, 1000)])
def test_two_arm_band(B, cells, K):
    """The band: both sides at delta / 2 from one simulation pass, equal to the
    one-sided calls at delta / 2, against the oracle; l0 <= R/K <= u0 and
    lower <= upper on every tile."""
    design = W.TWO_ARM
    tiles = W.two_arm_grid(cells, K)
    ctx = B.Context(design, K_max=K)
    dt = B.DeviceTiles(tiles)
    band = {k: v.clone() for k, v in ctx.validate_band(dt, -1.96, 0.02).items()}
    lo = {k: v.clone() for k, v in ctx.validate_lower(dt, -1.96, 0.01).items()}
    up = ctx.validate(dt, -1.96, 0.01)
    torch.cuda.synchronize()
    ctx.sync()
    assert torch.equal(band["R"], lo["R"]) and torch.equal(band["R"], up["R"])
    assert torch.equal(band["lower"], lo["lower"]) and torch.equal(band["l0"], lo["l0"])
    assert torch.equal(band["upper"], up["bound"]) and torch.equal(band["u0"], up["u0"])
    R = _np(band["R"])
    frac = R / tiles.K
    assert np.all(_np(band["l0"]) <= frac) and np.all(frac <= _np(band["u0"]))
    assert np.all(_np(band["lower"]) <= _np(band["upper"]))
    ref = O.simulate(design, tiles, -1.96)
    assert np.array_equal(R, ref["R"])
    _check_lower(lo, O.validate_lower(design, tiles, ref["R"], 0.01))
    refu = O.validate_bounds(design, tiles, ref["R"], 0.01)
    assert np.allclose(_np(band["upper"]), refu["bound"], rtol=RTOL, atol=0)


def test_plain_path_lower(B):
    design = W.TWO_ARM
    tiles = W.two_arm_grid(16, 2048)
    ctx = B.Context(design, K_max=2048)
    dt = B.DeviceTiles(tiles)
    a = {k: v.clone() for k, v in ctx.validate_lower(dt, -1.96, 0.01).items()}
    ctx.set_option(B.OPT_PLAIN, 1)
    b = ctx.validate_lower(dt, -1.96, 0.01)
    torch.cuda.synchronize()
    ctx.sync()
    assert torch.equal(a["R"], b["R"])
    assert np.allclose(_np(a["l0"]), _np(b["l0"]), rtol=RTOL, atol=0)
    la, lb = _np(a["lower"]), _np(b["lower"])
    assert np.all(np.abs(la - lb) <= RTOL * (1.0 - lb) + 1e-300)


def test_invalid_delta_raises(B):
    tiles = W.one_arm_tiles(4, 64)
    ctx = B.Context(W.ONE_ARM, K_max=64)
    dt = B.DeviceTiles(tiles)
    for bad in (0.0, 1.0, -0.1):
        with pytest.raises(B.CseError):
            ctx.validate_lower(dt, -1.96, bad)
        with pytest.raises(B.CseError):
            ctx.validate_band(dt, -1.96, bad)
