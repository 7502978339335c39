"""Path sharding over ranks (the data-parallel split of one optimisation), on
CPU: gloo ranks, the FP64 oracle as each rank's compute.

The estimate of Eq. 19 and the gradient of Eq. 21 are sums over independent
paths whose random streams depend on the path id only.  So the shards that
driver.shard_range gives, each normalised by the total count and summed by
driver.allreduce_sum, must reproduce one process's images; and the residual
taken from the summed images, fed to every rank's gradient of its own paths,
must sum to one process's gradient.  These are the two exchanges of
ShardedReconstruction's step (images before the residual, gradient before
Adam); a wrong normaliser, an overlapping or missing shard, or a residual
taken from a rank's partial images fails the comparison.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2110_00085_gb300.driver import shard_range


@pytest.mark.parametrize("n", [1, 2, 7, 10, 4096, (1 << 24) + 3])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_ranges_tile_the_budget(n, world):
    if n < world:
        pytest.skip("fewer paths than ranks")
    pos = 0
    counts = []
    for r in range(world):
        first, count = shard_range(n, r, world)
        assert first == pos
        pos += count
        counts.append(count)
    assert pos == n
    assert max(counts) - min(counts) <= 1 and min(counts) >= 1


def test_shard_range_rejects_bad_ranks():
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)
    with pytest.raises(ValueError):
        shard_range(10, 0, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _scene():
    from paper_2110_00085_gb300 import synth
    sc = synth.config(2, n_paths=1 << 9)       # 64^3 blobs in air: two particle types
    rng = np.random.default_rng(8)
    bt = (sc.beta_cloud * rng.uniform(0.8, 1.2, size=sc.beta_cloud.shape)).astype(np.float32)
    gt = np.random.default_rng(9).uniform(0.0, 1e-3, size=sc.n_pixels)
    return sc, bt, gt


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as td
    import oracle as O
    from paper_2110_00085_gb300.driver import allreduce_sum
    td.init_process_group("gloo", rank=rank, world_size=world)
    sc, bt, gt = _scene()
    n = sc.n_paths
    first, count = shard_range(n, rank, world)
    img = torch.from_numpy(O.render(sc, sc.beta_cloud, bt, first=first, n=count, n_norm=n)["images"])
    allreduce_sum(img)
    dldi = img.numpy() - gt                      # the residual of the summed images, the same on every rank
    g = torch.from_numpy(O.render(sc, sc.beta_cloud, bt, first=first, n=count, n_norm=n, dldi=dldi)["grad"])
    allreduce_sum(g)
    out[rank] = (img.numpy().copy(), g.numpy().copy())
    td.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_images_and_gradient_equal_one_process(world):
    import oracle as O
    sc, bt, gt = _scene()
    n = sc.n_paths
    one = O.render(sc, sc.beta_cloud, bt, grad_abs=True)
    ref = O.render(sc, sc.beta_cloud, bt, dldi=one["images"] - gt, grad_abs=True)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert sorted(out.keys()) == list(range(world))
    for r in range(world):
        img, g = out[r]
        # every rank holds the same bits after the all-reduce
        assert np.array_equal(img, out[0][0]) and np.array_equal(g, out[0][1])
    img, g = out[0]
    assert ref["images"].max() > 0 and np.abs(ref["grad"]).max() > 0
    # the same FP64 terms summed in another order
    assert np.all(np.abs(img - ref["images"]) <= 1e-12 * np.abs(ref["images"]) + 1e-300)
    assert np.all(np.abs(g - ref["grad"]) <= 1e-12 * ref["grad_abs"] + 1e-300)
    # a rank's own shard is not the whole estimate: the exchange is needed
    f0, c0 = shard_range(n, 0, world)
    part = O.render(sc, sc.beta_cloud, bt, first=f0, n=c0, n_norm=n)["images"]
    assert np.abs(part - ref["images"]).sum() > 0.2 * ref["images"].sum()
