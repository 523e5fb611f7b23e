"""GPU vs oracle parity for the one- and two-arm z-test designs, through the C ABI.

Integers (reject counts, success sums, order-statistic indices, the statistic
values selected as lambda) must match bit for bit; FP64 bounds, alpha' and the
score within 1e-12 relative.
"""
import math

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


def _check_sim(out, ref, d, K):
    assert np.array_equal(_np(out["R"]), ref["R"])
    assert np.array_equal(_np(out["Xrej"]), ref["Xrej"])
    sc = _np(out["score"])
    tol = 1e-12 * np.maximum(1.0, np.abs(ref["Xrej"]).astype(float))
    assert np.all(np.abs(sc - ref["score"]) <= tol)


def _check_bounds(out, ref):
    assert np.allclose(_np(out["u0"]), ref["u0"], rtol=RTOL, atol=0)
    assert np.allclose(_np(out["bound"]), ref["bound"], rtol=RTOL, atol=0)
    # q* is an argmin: where the bound is within 1e-3 of 1 (u0 near 1, R near K)
    # the objective is flat to FP64 rounding over a q-interval of relative width
    # ~1e-5, so q* is compared where the minimum is well conditioned and, beyond,
    # only checked to be an equally finite q >= 1 (the bound itself is compared
    # to 1e-12 above everywhere).
    q, qr = _np(out["qstar"]), ref["qstar"]
    assert np.array_equal(np.isinf(q), np.isinf(qr))
    fin = ~np.isinf(qr)
    assert np.all(q[fin] >= 1.0)
    sharp = fin & (ref["bound"] < 0.999)
    assert np.all(np.abs(q[sharp] - qr[sharp]) <= 1e-6 * np.abs(qr[sharp]))


def test_one_arm_full_config_validation(B):
    design, tiles = W.CONFIGS["c1"]()
    ctx = B.Context(design, K_max=tiles.K_max)
    dt = B.DeviceTiles(tiles)
    out = ctx.validate(dt, -1.96, 0.01)
    torch.cuda.synchronize()
    ctx.sync()
    ref = O.simulate(design, tiles, -1.96)
    _check_sim(out, ref, 1, tiles.K)
    _check_bounds(out, O.validate_bounds(design, tiles, ref["R"], 0.01))
    # tiles reject only when X >= 32
    assert np.all(_np(out["R"]) <= tiles.K)


@pytest.mark.parametrize("cells,K", [(16, 1000), (32, 2048), (8, 4099)])
def test_two_arm_grid_step(B, cells, K):
    design = W.TWO_ARM
    tiles = W.two_arm_grid(cells, K)
    ctx = B.Context(design, K_max=K)
    dt = B.DeviceTiles(tiles)
    out = ctx.step(dt, -1.96, 0.01, 0.025)
    torch.cuda.synchronize()
    ctx.sync()
    ref = O.simulate(design, tiles, -1.96)
    _check_sim(out, ref, 2, tiles.K)
    _check_bounds(out, O.validate_bounds(design, tiles, ref["R"], 0.01))
    cal = O.calibrate(design, tiles, 0.025)
    assert np.allclose(_np(out["alpha_prime"]), cal["alpha_prime"], rtol=RTOL, atol=0)
    assert np.array_equal(_np(out["lambda_tile"]), cal["lambda_tile"])
    assert out["lam"].item() == cal["lam"]


def test_calibrate_entry_point_and_ragged_K(B):
    design = W.TWO_ARM
    base = W.two_arm_grid(8, 1)
    rng = np.random.default_rng(3)
    tiles = base.with_K(rng.integers(1, 3001, size=base.n_tiles))   # ragged K, includes tiny K
    tiles.K[0] = 1
    ctx = B.Context(design, K_max=4096)
    dt = B.DeviceTiles(tiles)
    cal = ctx.calibrate(dt, 0.05)
    ref = O.calibrate(design, tiles, 0.05)
    assert np.allclose(_np(cal["alpha_prime"]), ref["alpha_prime"], rtol=RTOL, atol=0)
    assert np.array_equal(_np(cal["lambda_tile"]), ref["lambda_tile"])   # k = 0 gives -inf
    assert cal["lam"] == ref["lam"]
    sim = ctx.simulate_tiles(dt, -1.5)
    torch.cuda.synchronize()
    r = O.simulate(design, tiles, -1.5)
    assert np.array_equal(_np(sim[0]), r["R"]) and np.array_equal(_np(sim[1]), r["Xrej"])


def test_clopper_pearson_across_R_and_K(B):
    """Reject counts from 0 to K and ragged K up to 2^16: ~1,500 distinct (K, R)
    keys, more than the one-warp-per-key slots, so both roles of the distinct-key
    solve run (a warp per key first, a thread per key after)."""
    design = W.ONE_ARM
    rng = np.random.default_rng(11)
    n = 1500
    c = np.linspace(-0.5, 2.0, n)[:, None]   # P(reject) from ~0 to ~1
    h = np.full_like(c, 1.25 / n)
    K = rng.integers(1, 4097, size=n).astype(np.int32)
    big = rng.choice(n, size=24, replace=False)
    K[big] = rng.integers(4097, (1 << 16) + 1, size=24)
    K[:3] = [1, 2, 1 << 16]
    tiles = W.from_centers(c, h, np.ones(n, dtype=np.uint32), K)
    ctx = B.Context(design, K_max=1 << 16)
    out = ctx.validate(B.DeviceTiles(tiles), -1.96, 0.01)
    torch.cuda.synchronize()
    ctx.sync()
    ref = O.simulate(design, tiles, -1.96)
    _check_sim(out, ref, 1, tiles.K)
    R = ref["R"]
    assert (R == 0).any() and (R == tiles.K).any() and len(set(zip(K.tolist(), R.tolist()))) > 1400
    _check_bounds(out, O.validate_bounds(design, tiles, R, 0.01))


def test_adaptive_batch_small(B):
    design = W.TWO_ARM
    tiles = W.two_arm_adaptive(n_tiles=600, seed=5, log2K=(8, 9, 10, 11))
    ctx = B.Context(design, K_max=tiles.K_max)
    dt = B.DeviceTiles(tiles)
    out = ctx.step(dt, -1.96, 0.01, 0.025)
    torch.cuda.synchronize()
    ctx.sync()
    ref = O.simulate(design, tiles, -1.96)
    _check_sim(out, ref, 2, tiles.K)
    _check_bounds(out, O.validate_bounds(design, tiles, ref["R"], 0.01))
    cal = O.calibrate(design, tiles, 0.025)
    assert np.array_equal(_np(out["lambda_tile"]), cal["lambda_tile"])


@pytest.mark.parametrize("cfg", ["c2", "c3"])
def test_full_size_configs_sampled(B, cfg):
    """Full-size workload in the benchmark's launch configuration; sampled tiles
    recomputed one by one by the oracle."""
    design, tiles = W.CONFIGS[cfg]()
    ctx = B.Context(design, K_max=tiles.K_max)
    dt = B.DeviceTiles(tiles)
    out = ctx.step(dt, -1.96, 0.01, 0.025)
    torch.cuda.synchronize()
    ctx.sync()
    rng = np.random.default_rng(11)
    # sample: the tiles with the most rejections, the global-min tile, random ones
    R = _np(out["R"])
    lt = _np(out["lambda_tile"])
    rows = np.unique(np.concatenate([np.argsort(R)[-3:], [int(np.argmin(lt))],
                                     rng.choice(tiles.n_tiles, 6, replace=False)]))
    sub = tiles.subset(rows)
    ref = O.simulate(design, sub, -1.96)
    assert np.array_equal(R[rows], ref["R"])
    assert np.array_equal(_np(out["Xrej"])[rows], ref["Xrej"])
    vb = O.validate_bounds(design, sub, ref["R"], 0.01)
    assert np.allclose(_np(out["bound"])[rows], vb["bound"], rtol=RTOL, atol=0)
    cal = O.calibrate(design, sub, 0.025)
    assert np.array_equal(lt[rows], cal["lambda_tile"])
    assert np.allclose(_np(out["alpha_prime"])[rows], cal["alpha_prime"], rtol=RTOL, atol=0)
    # properties at any size: lambda* is the minimum; bounds >= CP >= R/K
    assert out["lam"].item() == lt.min()
    u0, b = _np(out["u0"]), _np(out["bound"])
    assert np.all(b >= u0 * (1 - 1e-15)) and np.all(u0 >= R / tiles.K)


def test_backward_matches_oracle(B):
    design = W.TWO_ARM
    tiles = W.two_arm_grid(16, 2000)
    ctx = B.Context(design, K_max=2048)
    theta = torch.tensor(tiles.centers, dtype=torch.float64, device="cuda", requires_grad=True)
    f = B.TypeIError.apply(theta, ctx, 1, 2000, -1.96)
    g = torch.linspace(0.5, 1.5, tiles.n_tiles, dtype=torch.float64, device="cuda")
    (f * g).sum().backward()
    ref = O.simulate(design, tiles, -1.96)
    assert np.array_equal(_np(f), ref["R"] / 2000.0)
    gr = O.score_backward(_np(g), ref["score"], tiles.K)
    assert np.allclose(_np(theta.grad), gr, rtol=1e-12, atol=1e-13)


def test_invalid_calls_raise(B):
    design = W.TWO_ARM
    tiles = W.two_arm_grid(4, 100)
    ctx = B.Context(design, K_max=128)
    dt = B.DeviceTiles(tiles)
    with pytest.raises(B.CseError):
        ctx.validate(dt, -1.96, 1.5)
    with pytest.raises(B.CseError):
        ctx.calibrate(dt, 0.0)
    big = B.DeviceTiles(tiles.with_K(200))   # K_max of the set above the context's
    with pytest.raises(B.CseError):
        ctx.simulate_tiles(big, -1.96)


def test_tiles_without_hypothesis_or_negative_width_are_reported(B):
    """A tile that meets no null hypothesis, or has a negative (or NaN) half-width,
    fails the device-side check: its bounds are NaN, the other tiles' are those
    of a clean run, cse_sync reports DEVICE_CHECK once and then clears it."""
    design = W.TWO_ARM
    tiles = W.two_arm_grid(8, 256)
    ctx = B.Context(design, K_max=256)
    clean = ctx.validate(B.DeviceTiles(tiles), -1.96, 0.01)
    torch.cuda.synchronize()
    ctx.sync()
    clean_b = clean["bound"].cpu().numpy().copy()
    bad = tiles.subset(np.arange(tiles.n_tiles))
    bad.null_mask[2] = 0
    bad.halfwidth[5, 1] = -0.1
    bad.halfwidth[7, 0] = np.nan
    out = ctx.validate(B.DeviceTiles(bad), -1.96, 0.01)
    torch.cuda.synchronize()
    with pytest.raises(B.CseError) as e:
        ctx.sync()
    assert e.value.status == -6
    b = out["bound"].cpu().numpy()
    flagged = np.zeros(tiles.n_tiles, dtype=bool)
    flagged[[2, 5, 7]] = True
    assert np.all(np.isnan(b[flagged]))
    assert np.array_equal(b[~flagged], clean_b[~flagged])
    ctx.sync()   # cleared


@pytest.mark.parametrize("cells,K", [(16, 3000), (32, 2048)])
def test_plain_path_gives_the_same_results(B, cells, K):
    """The plain comparison path (per-(tile, sim) binary search counts, FP64-only
    bound pass) reproduces the chosen path: integers exactly, FP64 to 1e-12."""
    design = W.TWO_ARM
    tiles = W.two_arm_grid(cells, K)
    ctx = B.Context(design, K_max=K)
    dt = B.DeviceTiles(tiles)
    a = {k: v.clone() for k, v in ctx.step(dt, -1.96, 0.01, 0.025).items()}
    ctx.set_option(B.OPT_PLAIN, 1)
    b = ctx.step(dt, -1.96, 0.01, 0.025)
    torch.cuda.synchronize()
    ctx.sync()
    for key in ("R", "Xrej", "lambda_tile", "lam"):
        assert torch.equal(a[key], b[key]), key
    for key in ("score", "u0", "bound", "alpha_prime"):
        assert np.allclose(_np(a[key]), _np(b[key]), rtol=RTOL, atol=0), key
    ref = O.simulate(design, tiles, -1.96)
    assert np.array_equal(_np(b["R"]), ref["R"])


def test_cuda_graph_replay_and_autotune(B):
    """A step captured in a CUDA graph replays to the same outputs as direct
    calls; the autotuner's choice of block size leaves results unchanged."""
    design = W.TWO_ARM
    tiles = W.two_arm_grid(32, 3000)
    ctx = B.Context(design, K_max=3000)
    dt = B.DeviceTiles(tiles)
    ref = {k: v.clone() for k, v in ctx.step(dt, -1.96, 0.01, 0.025).items()}
    ones = torch.ones(tiles.n_tiles, dtype=torch.float64, device="cuda")
    out = ctx.step_buffers(dt)
    g = B.StepGraph(ctx, dt, -1.96, 0.01, 0.025, design.seed, out, ones)
    for _ in range(2):
        o, grad = g.replay()
        torch.cuda.synchronize()
        for key in ("R", "Xrej", "lambda_tile", "lam", "bound", "u0", "alpha_prime", "score"):
            assert torch.equal(o[key], ref[key]), key
    threads, tiles_pb = ctx.autotune(dt, -1.96, 0.025)
    assert (threads, tiles_pb) in ((128, 1), (256, 1), (512, 1), (64, 1), (128, 2), (256, 2), (256, 4))
    again = ctx.step(dt, -1.96, 0.01, 0.025)
    torch.cuda.synchronize()
    for key in ("R", "Xrej", "lambda_tile", "lam"):
        assert torch.equal(again[key], ref[key]), key


def test_reseed_takes_effect_at_the_next_call(B):
    """cse_reseed only records the key; the next simulating call regenerates the
    uniforms.  The last of several reseeds wins, and the counts match the oracle
    at that key."""
    import dataclasses
    tiles = W.two_arm_grid(8, 1024)
    ctx = B.Context(W.TWO_ARM, seed=5, K_max=1024)
    dt = B.DeviceTiles(tiles)
    r5 = _np(ctx.simulate_tiles(dt, -1.96)[0]).copy()
    ctx.reseed(123)
    ctx.reseed(77)
    r77 = _np(ctx.simulate_tiles(dt, -1.96)[0]).copy()
    torch.cuda.synchronize()
    ctx.sync()
    assert np.array_equal(r5, O.simulate(dataclasses.replace(W.TWO_ARM, seed=5), tiles, -1.96)["R"])
    assert np.array_equal(r77, O.simulate(dataclasses.replace(W.TWO_ARM, seed=77), tiles, -1.96)["R"])
    assert not np.array_equal(r5, r77)
    ctx.reseed(5)
    assert np.array_equal(_np(ctx.simulate_tiles(dt, -1.96)[0]), r5)


def test_profile_only_times_one_kernel_group(B):
    """cse_profile_only restricts the event timing to one kernel group (the
    others launch without events); NULL times all groups again; an unknown name
    is refused.  Outputs do not depend on the profiler."""
    tiles = W.two_arm_grid(16, 2048)
    ctx = B.Context(W.TWO_ARM, K_max=2048)
    dt = B.DeviceTiles(tiles)
    ref = {k: v.clone() for k, v in ctx.step(dt, -1.96, 0.01, 0.025).items()}
    ctx.profile(True, only="sim_ztest")
    ctx.profile_read()
    o = ctx.step(dt, -1.96, 0.01, 0.025)
    one = ctx.profile_read()
    assert set(one) == {"sim_ztest"} and one["sim_ztest"][0] == 1 and one["sim_ztest"][1] > 0.0
    for key in ("R", "lambda_tile", "lam", "bound", "alpha_prime"):
        assert torch.equal(o[key], ref[key]), key
    ctx.profile(True)
    ctx.step(dt, -1.96, 0.01, 0.025)
    every = ctx.profile_read()
    assert {"sim_ztest", "alpha_prime", "bounds", "axis_counts"} <= set(every)
    with pytest.raises(B.CseError):
        ctx.profile(True, only="no_such_kernel")
    ctx.profile(False)


@pytest.mark.parametrize("box", [101, 700])
def test_box_slabs_give_the_same_results(B, box):
    """A tile box larger than the histogram capacity is done in slabs of whole
    rows (one pass over the sims per slab): with the capacity set below the
    boxes of this grid (one row per slab at 101 cells), every output of a step,
    the randomised tie pass's r* and m included, equals the one-pass results,
    and R matches the oracle."""
    tiles = W.two_arm_grid(16, 3000)
    ctx = B.Context(W.TWO_ARM, seed=21, K_max=3000)
    dt = B.DeviceTiles(tiles)
    ref = {k: v.clone() for k, v in ctx.step(dt, -1.96, 0.01, 0.025).items()}
    rr = ctx.calibrate_rand(dt, 0.025)
    torch.cuda.synchronize()
    ctx.set_option(B.OPT_CELLS_BOX, box)
    got = ctx.step(dt, -1.96, 0.01, 0.025)
    gr = ctx.calibrate_rand(dt, 0.025)
    torch.cuda.synchronize()
    for key in ("R", "Xrej", "score", "lambda_tile", "lam", "bound", "alpha_prime"):
        assert torch.equal(got[key], ref[key]), key
    for key, a in rr.items():
        assert (torch.equal(a, gr[key]) if isinstance(a, torch.Tensor) else a == gr[key]), key
    ctx.set_option(B.OPT_CELLS_BOX, 0)
    import dataclasses
    assert np.array_equal(_np(got["R"]), O.simulate(dataclasses.replace(W.TWO_ARM, seed=21), tiles, -1.96)["R"])
    with pytest.raises(B.CseError):
        ctx.set_option(B.OPT_CELLS_BOX, 100)     # shorter than a row
    with pytest.raises(B.CseError):
        ctx.set_option(B.OPT_CELLS_BOX, 5000)    # above the allocated capacity


def test_programmatic_dependent_launch_changes_nothing(B):
    """The step's kernels give the same outputs with and without programmatic
    dependent launch, directly and replayed from a CUDA graph."""
    tiles = W.two_arm_grid(32, 2048)
    ctx = B.Context(W.TWO_ARM, seed=3, K_max=2048)
    dt = B.DeviceTiles(tiles)
    ctx.set_option(B.OPT_PDL, 0)
    ref = {k: v.clone() for k, v in ctx.step(dt, -1.96, 0.01, 0.025).items()}
    band0 = {k: v.clone() for k, v in ctx.validate_band(dt, -1.96, 0.02).items()}
    ctx.set_option(B.OPT_PDL, 1)
    got = ctx.step(dt, -1.96, 0.01, 0.025)
    band1 = ctx.validate_band(dt, -1.96, 0.02)
    torch.cuda.synchronize()
    for key in ("R", "Xrej", "score", "lambda_tile", "lam", "bound", "u0", "alpha_prime"):
        assert torch.equal(got[key], ref[key]), key
    for key, v in band0.items():
        assert torch.equal(band1[key], v), key
    ones = torch.ones(tiles.n_tiles, dtype=torch.float64, device="cuda")
    g = B.StepGraph(ctx, dt, -1.96, 0.01, 0.025, 3, ctx.step_buffers(dt), ones)
    o, _ = g.replay()
    torch.cuda.synchronize()
    for key in ("R", "lambda_tile", "lam", "bound"):
        assert torch.equal(o[key], ref[key]), key
    with pytest.raises(B.CseError):
        ctx.set_option(B.OPT_PDL, 2)


@pytest.mark.parametrize("which", ["one_arm", "two_arm"])
def test_selection_on_the_gpus_own_statistics(B, which):
    """lambda_i of the fused step is the k_i-th smallest of the GPU's own per-sim
    statistics (cse_statistics), k_i = floor((K_i + 1) alpha'_i) from the GPU's
    alpha' (Eq. calibrated-threshold): checked with np.sort and by counting, on
    ragged K including k_i = 0.  Independent of the oracle's selection; the
    exported statistics also equal the oracle's value for value."""
    if which == "one_arm":
        design = W.ONE_ARM
        rng = np.random.default_rng(2)
        n = 96
        c = np.linspace(-0.45, 0.25, n)[:, None]
        K = rng.integers(40, 3000, size=n).astype(np.int32)
        K[:4] = [1, 3, 39, 41]
        tiles = W.from_centers(c, np.full_like(c, 0.01), np.ones(n, dtype=np.uint32), K)
        lam = -1.96
    else:
        design = W.TWO_ARM
        base = W.two_arm_grid(12, 1, lo=-1.0, hi=1.0)
        rng = np.random.default_rng(4)
        K = rng.integers(1, 2500, size=base.n_tiles).astype(np.int32)
        K[:3] = [1, 5, 40]
        tiles = base.with_K(K)
        lam = -1.96
    ctx = B.Context(design, K_max=tiles.K_max)
    dt = B.DeviceTiles(tiles)
    out = ctx.step(dt, lam, 0.01, 0.025)
    S, off = ctx.statistics(dt)
    torch.cuda.synchronize()
    ctx.sync()
    S, off = _np(S), _np(off)
    ap, lt, R = _np(out["alpha_prime"]), _np(out["lambda_tile"]), _np(out["R"])
    k = np.minimum(np.floor((tiles.K + 1.0) * ap).astype(np.int64), tiles.K)
    ref = O.simulate(design, tiles, lam, want_S=True)
    edges = 0
    for i in range(tiles.n_tiles):
        Si = S[off[i]: off[i] + tiles.K[i]].astype(np.float64)
        assert np.array_equal(Si, ref["S"][i])
        assert R[i] == int((Si < lam).sum())
        if k[i] < 1:
            assert lt[i] == -math.inf
            continue
        srt = np.sort(Si)
        assert lt[i] == srt[k[i] - 1], (i, k[i])
        assert int((Si < lt[i]).sum()) < k[i] <= int((Si <= lt[i]).sum())
        edges += int(k[i] >= 2 and srt[k[i] - 2] != srt[k[i] - 1])
    assert (k == 0).any() and edges >= 5
    assert out["lam"].item() == lt.min()


def test_type1_error_entry_matches_the_tile_path(B):
    """cse_type1_error (points given by coordinates; distinct coordinates gathered
    on the device) gives the same R, score and f_hat = R / K as cse_simulate_tiles
    on the axis-indexed tile set of the same points, for points in any order,
    with repeated points, per-point K and a second call with fewer points on the
    grown scratch; the oracle agrees."""
    design = W.TWO_ARM
    tiles = W.two_arm_grid(16, 1)
    rng = np.random.default_rng(8)
    perm = rng.permutation(tiles.n_tiles)
    rows = np.concatenate([perm, perm[:7]])              # shuffled, with repeats
    sub = tiles.subset(rows).with_K(rng.integers(1, 3001, size=len(rows)))
    ctx = B.Context(design, K_max=3000)
    theta = torch.tensor(sub.centers, dtype=torch.float64, device="cuda")
    Kt = torch.tensor(sub.K, dtype=torch.int32, device="cuda")
    nm = torch.tensor(sub.null_mask.view(np.int32), device="cuda")
    fhat, R, G, _ = ctx.type1_error(theta, nm, Kt, -1.96)
    R2, X2, G2 = ctx.simulate_tiles(B.DeviceTiles(sub), -1.96)
    torch.cuda.synchronize()
    ctx.sync()
    assert torch.equal(R, R2)
    assert np.allclose(_np(G), _np(G2), rtol=1e-12, atol=1e-12)
    assert np.array_equal(_np(fhat), _np(R) / sub.K)      # one correctly rounded division
    ref = O.simulate(design, sub, -1.96)
    assert np.array_equal(_np(R), ref["R"])
    few = sub.subset(np.arange(20))
    f2, r2, _, _ = ctx.type1_error(torch.tensor(few.centers, dtype=torch.float64, device="cuda"),
                                   torch.tensor(few.null_mask.view(np.int32), device="cuda"),
                                   torch.tensor(few.K, dtype=torch.int32, device="cuda"), -1.96)
    torch.cuda.synchronize()
    assert np.array_equal(_np(r2), ref["R"][:20])
    with pytest.raises(B.CseError):
        ctx.type1_error(theta, nm, 4000, -1.96)          # K_max above the context's


def test_cuda_graph_replay_of_a_mixed_batch(B):
    """The batching row at a testable size: tiles of four widths (h = 2^-4..2^-7)
    and five K (2^8..2^12) in one persistent launch, the whole step captured in
    a CUDA graph.  Two replays equal the eager step exactly, and sampled tiles
    equal the oracle."""
    design = W.TWO_ARM
    tiles = W.two_arm_adaptive(n_tiles=4000, seed=12, log2K=(8, 9, 10, 11, 12))
    assert len(np.unique(tiles.halfwidth[:, 0])) == 4 and len(np.unique(tiles.K)) == 5
    ctx = B.Context(design, seed=77, K_max=tiles.K_max)
    dt = B.DeviceTiles(tiles)
    ref = {k: v.clone() for k, v in ctx.step(dt, -1.96, 0.01, 0.025).items()}
    ones = torch.ones(tiles.n_tiles, dtype=torch.float64, device="cuda")
    g_ref = B.score_backward(ones, ref["score"], dt.K).clone()
    out = ctx.step_buffers(dt)
    g = B.StepGraph(ctx, dt, -1.96, 0.01, 0.025, 77, out, ones)
    for _ in range(2):
        for v in out.values():
            v.zero_()
        o, grad = g.replay()
        torch.cuda.synchronize()
        for key in ("R", "Xrej", "score", "lambda_tile", "lam", "bound", "u0", "qstar", "alpha_prime"):
            assert torch.equal(o[key], ref[key]), key
        assert torch.equal(grad, g_ref)
    import dataclasses
    rows = np.random.default_rng(4).choice(tiles.n_tiles, 30, replace=False)
    sub = tiles.subset(rows)
    d77 = dataclasses.replace(design, seed=77)
    r = O.simulate(d77, sub, -1.96)
    assert np.array_equal(_np(ref["R"])[rows], r["R"])
    assert np.array_equal(_np(ref["Xrej"])[rows], r["Xrej"])
    cal = O.calibrate(d77, sub, 0.025)
    assert np.array_equal(_np(ref["lambda_tile"])[rows], cal["lambda_tile"])
    vb = O.validate_bounds(d77, sub, r["R"], 0.01)
    assert np.allclose(_np(ref["bound"])[rows], vb["bound"], rtol=RTOL, atol=0)


@pytest.mark.parametrize("threads,tiles_pb", [(64, 1), (128, 2), (256, 2), (256, 4), (512, 1)])
def test_cell_kernel_configurations_agree(B, threads, tiles_pb):
    """Every (threads per block, tiles per block) configuration of the z-test
    cell kernel gives the step's outputs bit for bit, on a mixed batch (uneven
    widths and K) including slab boxes; the two-arm oracle agrees on R."""
    tiles = W.two_arm_adaptive(n_tiles=1500, seed=3, log2K=(9, 10, 11, 12))
    ctx = B.Context(W.TWO_ARM, seed=8, K_max=tiles.K_max)
    dt = B.DeviceTiles(tiles)
    ref = {k: v.clone() for k, v in ctx.step(dt, -1.96, 0.01, 0.025).items()}
    rr = ctx.calibrate_rand(dt, 0.025)
    ctx.set_option(B.OPT_SIM_THREADS, threads)
    ctx.set_option(B.OPT_SIM_TILES, tiles_pb)
    got = ctx.step(dt, -1.96, 0.01, 0.025)
    gr = ctx.calibrate_rand(dt, 0.025)
    torch.cuda.synchronize()
    ctx.sync()
    for key in ("R", "Xrej", "score", "lambda_tile", "lam", "bound", "alpha_prime"):
        assert torch.equal(got[key], ref[key]), key
    for key, a in rr.items():
        assert (torch.equal(a, gr[key]) if isinstance(a, torch.Tensor) else a == gr[key]), key
    ctx.set_option(B.OPT_CELLS_BOX, 202)          # two rows per slab: the slab path in groups
    sl = ctx.step(dt, -1.96, 0.01, 0.025)
    torch.cuda.synchronize()
    for key in ("R", "Xrej", "lambda_tile", "lam"):
        assert torch.equal(sl[key], ref[key]), key
    import dataclasses
    assert np.array_equal(_np(got["R"]), O.simulate(dataclasses.replace(W.TWO_ARM, seed=8), tiles, -1.96)["R"])
    with pytest.raises(B.CseError):
        ctx.set_option(B.OPT_SIM_TILES, 3)


@pytest.mark.gpu
def test_step_memo_keys_match_the_validation_path(B):
    """In cse_step the cell kernel inserts each tile's (K, R) into the
    Clopper-Pearson memo; cse_validate marks the keys with k_cp_mark.  Both give
    the same counts and the same u0, bit for bit, on a batch of mixed K."""
    tiles = W.two_arm_adaptive(n_tiles=3000, seed=12, log2K=(9, 10, 11))
    ctx = B.Context(W.TWO_ARM, seed=3, K_max=tiles.K_max)
    dt = B.DeviceTiles(tiles)
    a = {k: v.clone() for k, v in ctx.step(dt, -1.96, 0.01, 0.025).items()}
    v = ctx.validate(dt, -1.96, 0.01)
    torch.cuda.synchronize()
    ctx.sync()
    assert torch.equal(v["R"], a["R"]) and torch.equal(v["Xrej"], a["Xrej"])
    assert torch.equal(v["u0"], a["u0"])
    assert np.allclose(_np(v["bound"]), _np(a["bound"]), rtol=1e-14, atol=0)
