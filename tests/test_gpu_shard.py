"""ShardedReconstruction on the GPU: two gloo ranks, each a process on the
same device (their kernels never wait on each other; the all-reduces run on
the host side of gloo), against Reconstruction in one process.

Every event's contribution is computed from its own stored path alone, so a
rank's events give the same FP32 terms as in one process: the summed images
equal one process's to FP64 summation order.  The gradient's same-voxel
pre-sums inside a warp group other neighbours when the events are binned per
shard, so it agrees to FP32 rounding of those partial sums."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2110_00085_gb300 import native as N
from paper_2110_00085_gb300 import synth
from paper_2110_00085_gb300.driver import Reconstruction, ShardedReconstruction

pytestmark = pytest.mark.gpu

STEPS = 3
N_R = 2          # step 3 resamples: the shards are stored twice


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _spec():
    return synth.config(1, n_paths=(1 << 14) + 5)     # a budget that 2 ranks split unevenly after halving


def _run(rec, steps):
    out = []
    for _ in range(steps):
        rec.step()
        torch.cuda.synchronize()
        out.append((rec.images.cpu().numpy().copy(), rec.grad.cpu().numpy().copy(), rec.beta.cpu().numpy().copy(),
                    float(rec.loss.item())))
    return out


def _worker(rank, world, port, gt, beta0, kw, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as td
    torch.cuda.set_device(0)
    td.init_process_group("gloo", rank=rank, world_size=world)
    sc = _spec()
    scene = N.Scene(sc)
    rec = ShardedReconstruction(scene, torch.from_numpy(gt).cuda(), torch.from_numpy(beta0).cuda(), sc.n_paths,
                                n_r=N_R, seed=sc.seed, **kw)
    out[rank] = _run(rec, STEPS)
    rec.close()
    scene.close()
    td.destroy_process_group()


def _compare(kw):
    sc = _spec()
    scene = N.Scene(sc)
    beta_gt = torch.from_numpy(sc.beta_cloud.reshape(-1)).cuda()
    gt = scene.render_forward(beta_gt, 1 << 15, sc.seed + 99)
    beta0 = (0.8 * beta_gt).contiguous()
    rec = Reconstruction(scene, gt, beta0, sc.n_paths, n_r=N_R, seed=sc.seed, **kw)
    ref = _run(rec, STEPS)
    rec.close()
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), gt.cpu().numpy(), beta0.cpu().numpy(), kw, out),
                       nprocs=world, start_method="spawn", join=True)
    for r in range(1, world):
        for a, b in zip(out[0], out[r]):
            assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])), "ranks disagree after the all-reduce"
    scene.close()
    return ref, out[0]


def test_sharded_steps_equal_one_process_at_fixed_extinction():
    """lr = 0: the extinction stays put, so all three steps (two path sets,
    the second stored at step 3) compare element by element."""
    for dec in (False, True):
        ref, got = _compare(dict(lr=0.0, decorrelate=dec))
        for k, ((i1, g1, b1, l1), (i2, g2, b2, l2)) in enumerate(zip(ref, got)):
            assert i1.max() > 0 and np.abs(g1).max() > 0
            assert np.allclose(i2, i1, rtol=1e-12, atol=0), (dec, k)
            assert np.allclose(g2, g1, rtol=1e-5, atol=1e-7 * np.abs(g1).max()), (dec, k)
            assert np.array_equal(b2, b1)
            assert l2 == pytest.approx(l1, rel=1e-12)


def test_sharded_adam_step_moves_the_extinction_like_one_process():
    """lr > 0: after one step the extinction agrees wherever the gradient is
    resolved above the FP32 pre-sum noise (elsewhere Adam's first step,
    -lr sign(g), may take either sign)."""
    ref, got = _compare(dict(lr=0.5))
    _, g1, b1, _ = ref[0]
    _, _, b2, _ = got[0]
    firm = np.abs(g1) > 1e-4 * np.abs(g1).max()
    assert firm.sum() > 1000
    assert np.allclose(b2[firm], b1[firm], rtol=1e-6, atol=1e-6)
    assert np.abs(b1 - 0.8 * synth.config(1).beta_cloud.reshape(-1)).max() > 0.1


def _bench_rank(rank, world, port, out):
    import contextlib
    import io
    import sys
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK="0")
    import bench
    sys.argv = ["bench.py", "--gpus", str(world), "--steps", "2", "--warmup", "1", "--paths", str(1 << 16),
                "--no-cpu", "--no-calibration", "--shard", "--shard-backend", "gloo"]
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.main()
    out[rank] = buf.getvalue()


def test_bench_sharded_path_runs_on_two_ranks():
    """bench.py --shard end to end: two ranks (processes on this one GPU,
    gloo in place of NCCL, which needs a GPU per rank) time one optimisation
    of 2 x 2^16 paths; rank 0 prints the line, which counts every rank's
    paths and names the sharding."""
    import json
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_bench_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    lines = [l for l in out[0].splitlines() if l.startswith("{")]
    assert len(lines) == 1 and not [l for l in out[1].splitlines() if l.startswith("{")]
    d = json.loads(lines[0])
    assert d["n_gpus"] == world and d["config"]["n_paths"] == 1 << 16
    assert "sharded over 2 ranks" in d["config"]["parallelism"]
    assert d["value"] == pytest.approx(world * (1 << 16) / (d["ms_per_step"] * 1e-3), rel=1e-9)
    assert d["gpu_launches"] > 0 and d["matched_error"] is None
