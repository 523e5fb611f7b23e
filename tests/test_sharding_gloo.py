"""Multi-rank calibration on CPU: two gloo ranks, each calibrating its shard of a
platten with the oracle, then one all-reduce MIN; the result must equal the
unsharded run tile by tile and in the global threshold."""
import os
import pickle
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2212_10042_gb300 import sharding
from paper_2212_10042_gb300 import workloads as W


def _platten():
    base = W.two_arm_grid(8, 1)
    rng = np.random.default_rng(2)
    return W.TWO_ARM, base.with_K(rng.integers(200, 1200, size=base.n_tiles))


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    design, tiles = _platten()

    def shard_fn(lo, hi):
        return O.calibrate(design, tiles.subset(np.arange(lo, hi)), 0.05)["lambda_tile"]

    res = sharding.calibrate_sharded(shard_fn, tiles.K, rank, world)
    with open(os.path.join(outdir, "r%d.pkl" % rank), "wb") as f:
        pickle.dump(res, f)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_bounds_balance():
    K = np.array([10, 10, 10, 10, 100, 1, 1, 1])
    b = sharding.shard_bounds(K, 2)
    assert b[0][0] == 0 and b[-1][1] == len(K) and b[0][1] == b[1][0]
    assert sharding.shard_bounds(K, 1) == [(0, len(K))]
    b3 = sharding.shard_bounds(np.ones(10), 3)
    assert [hi - lo for lo, hi in b3] in ([3, 3, 4], [3, 4, 3], [4, 3, 3])
    # more ranks than tiles: empty ranges are allowed, coverage stays exact
    b = sharding.shard_bounds([5, 5], 4)
    assert sum(hi - lo for lo, hi in b) == 2


def test_two_rank_calibration_matches_unsharded():
    from oracle import oracle as O
    O.lib()
    design, tiles = _platten()
    ref = O.calibrate(design, tiles, 0.05)
    port = 29500 + (os.getpid() % 2000)
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, port, d), nprocs=2, join=True)
        res = [pickle.load(open(os.path.join(d, "r%d.pkl" % r), "rb")) for r in range(2)]
    lam_tile = np.concatenate([r[2] for r in res])
    assert res[0][0] == 0 and res[0][1] == res[1][0] and res[1][1] == tiles.n_tiles
    assert np.array_equal(lam_tile, ref["lambda_tile"])
    assert res[0][3] == res[1][3] == ref["lam"]
