"""The allocation-free entry point cse_simulate_tiles_static against cse_simulate_tiles.

Some callers cannot allocate device memory (a plugin inside a host program
that owns all GPU memory, or code that must not risk the device-wide
synchronisation of cudaMalloc).  cse_simulate_tiles_static serves them from a
fixed scratch array inside the library; this test checks, through the C ABI,
that two calls in a row give the same results as the context-based entry
point (integers bit for bit, the FP64 score within 1e-12), that calls after a
failed call or a call of another design are not affected by what those left in
the shared array, that a request beyond the fixed capacity is refused, and that
a capturing stream is refused.  The file is collected last.
"""
import numpy as np
import pytest
import torch

from paper_2212_10042_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2212_10042_gb300 import binding
    binding.lib()
    return binding


def _same(a, b):
    R0, X0, G0 = [t.cpu().numpy() for t in a]
    R1, X1, G1 = [t.cpu().numpy() for t in b]
    assert np.array_equal(R0, R1)
    assert np.array_equal(X0, X1)
    assert np.allclose(G0, G1, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("which", ["one_arm", "two_arm"])
def test_static_matches_context_twice(B, which):
    if which == "one_arm":
        design, tiles, lam, seed = W.ONE_ARM, W.one_arm_tiles(64, 8192), -1.96, 5
    else:
        design, tiles, lam, seed = W.TWO_ARM, W.two_arm_grid(24, 3001), -1.8, 11
    dt = B.DeviceTiles(tiles)
    ctx = B.Context(design, seed=seed, K_max=tiles.K_max)
    ref = ctx.simulate_tiles(dt, lam)
    torch.cuda.synchronize()
    ctx.sync()
    first = B.simulate_tiles_static(design, seed, dt, lam)
    second = B.simulate_tiles_static(design, seed, dt, lam)
    torch.cuda.synchronize()
    _same(ref, first)
    _same(ref, second)
    ctx.close()


def test_static_refuses_beyond_capacity(B):
    tiles = W.two_arm_grid(8, 65536)      # 2 x 65536 x 100 uniforms alone exceed 32 MiB
    dt = B.DeviceTiles(tiles)
    with pytest.raises(B.CseError) as e:
        B.simulate_tiles_static(W.TWO_ARM, 0, dt, -1.96)
    assert e.value.status == -7


def test_static_after_a_failed_call_and_across_designs(B):
    """Every call shares the fixed array and finds the previous call's contents
    in it.  A call whose tile has K_i above the set's K_max leaves the error flag
    set (DEVICE_CHECK); the next valid call must clear it and match the context
    path.  A two-arm call followed by a one-arm call with a smaller K_max (other
    table sizes, other count rows) must match the context path too."""
    tiles = W.two_arm_grid(16, 2048)
    dt = B.DeviceTiles(tiles)
    K_bad = dt.K.clone()
    K_bad[3] = 2049
    bad = B.DeviceTiles.from_tensors(dt.axis, dt.idx, dt.halfwidth, dt.null_mask, K_bad, 2048)
    with pytest.raises(B.CseError) as e:
        B.simulate_tiles_static(W.TWO_ARM, 9, bad, -1.96)
    assert e.value.status == -6
    ctx = B.Context(W.TWO_ARM, seed=9, K_max=2048)
    ref = ctx.simulate_tiles(dt, -1.96)
    torch.cuda.synchronize()
    ctx.sync()
    ctx.close()
    _same(ref, B.simulate_tiles_static(W.TWO_ARM, 9, dt, -1.96))

    one = W.one_arm_tiles(40, 700, lo=-1.0, hi=0.0)
    d1 = B.DeviceTiles(one)
    ctx1 = B.Context(W.ONE_ARM, seed=4, K_max=700)
    ref1 = ctx1.simulate_tiles(d1, -1.7)
    torch.cuda.synchronize()
    ctx1.sync()
    ctx1.close()
    _same(ref1, B.simulate_tiles_static(W.ONE_ARM, 4, d1, -1.7))
    _same(ref, B.simulate_tiles_static(W.TWO_ARM, 9, dt, -1.96))


def test_static_refuses_a_capturing_stream(B):
    """The call synchronises its stream, which a CUDA graph capture cannot hold:
    on a capturing stream it returns INVALID_ARG before any GPU work and the
    capture stays usable."""
    tiles = W.two_arm_grid(8, 512)
    dt = B.DeviceTiles(tiles)
    x = torch.zeros(4, device="cuda")
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=side):
        x.add_(1.0)
        with pytest.raises(B.CseError) as e:
            B.simulate_tiles_static(W.TWO_ARM, 0, dt, -1.96, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    assert e.value.status == -1
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(x, torch.ones(4, device="cuda"))
