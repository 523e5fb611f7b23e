"""The sharded calibration with the CUDA library: two gloo ranks on the one GPU,
each running cse_calibrate on its own tile range (balanced by sum K_i), then
one all-reduce MIN of lambda_i (Eq. calibrated-threshold-final).  The ranks'
kernels never wait on one another: each calibrates independently and the only
exchange is the host-side all-reduce.  Per-tile thresholds and the global
threshold must equal the unsharded GPU run and the oracle."""
import os
import pickle
import tempfile

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2212_10042_gb300 import sharding
from paper_2212_10042_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _platten():
    tiles = W.two_arm_adaptive(n_tiles=3000, seed=9, log2K=(9, 10, 11, 12))
    return W.TWO_ARM, tiles


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    from paper_2212_10042_gb300 import binding as B
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    design, tiles = _platten()
    ctx = B.Context(design, K_max=tiles.K_max)

    def shard_fn(lo, hi):
        dt = B.DeviceTiles(tiles.subset(np.arange(lo, hi)))
        return ctx.calibrate(dt, 0.025)["lambda_tile"].cpu().numpy()

    res = sharding.calibrate_sharded(shard_fn, tiles.K, rank, world)
    ctx.close()
    with open(os.path.join(outdir, "r%d.pkl" % rank), "wb") as f:
        pickle.dump(res, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gpu_calibration_matches_unsharded():
    from oracle import oracle as O
    from paper_2212_10042_gb300 import binding as B
    B.lib()
    design, tiles = _platten()
    ctx = B.Context(design, K_max=tiles.K_max)
    whole = ctx.calibrate(B.DeviceTiles(tiles), 0.025)
    lam_whole = whole["lambda_tile"].cpu().numpy()
    ctx.close()
    port = 31500 + (os.getpid() % 2000)
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, port, d), nprocs=2, join=True)
        res = [pickle.load(open(os.path.join(d, "r%d.pkl" % r), "rb")) for r in range(2)]
    assert res[0][0] == 0 and res[0][1] == res[1][0] and res[1][1] == tiles.n_tiles
    lam_tile = np.concatenate([r[2] for r in res])
    assert np.array_equal(lam_tile, lam_whole)
    assert res[0][3] == res[1][3] == whole["lam"] == lam_whole.min()
    rows = np.random.default_rng(1).choice(tiles.n_tiles, 40, replace=False)
    ref = O.calibrate(design, tiles.subset(rows), 0.025)
    assert np.array_equal(lam_tile[rows], ref["lambda_tile"])
