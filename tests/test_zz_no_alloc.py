"""The allocation-free entry point cse_simulate_tiles_static against cse_simulate_tiles.

Some callers cannot allocate device memory (a plugin inside a host program
that owns all GPU memory, or code that must not risk the device-wide
synchronisation of cudaMalloc).  cse_simulate_tiles_static serves them from a
fixed scratch array inside the library; this test checks, through the C ABI,
that two calls in a row give the same results as the context-based entry
point (integers bit for bit, the FP64 score within 1e-12), and that a request
beyond the fixed capacity is refused.  The file is collected last.
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
