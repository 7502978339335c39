"""Batched launches: several scenes of uneven size in one launch per pass
(persistent or grouped schedule, or the per-scene sequence) give the
per-scene results and match the oracle; a captured CUDA graph of the step
replays the eager step, across a resample."""
import numpy as np
import pytest
import torch

from paper_2110_00085_gb300 import native as N
from paper_2110_00085_gb300 import synth
from paper_2110_00085_gb300.driver import BatchReconstruction
from paper_2110_00085_gb300.tune import tune_blocks

import oracle as O
from _parity import (MAX_DIVERGENT, assert_grad_close, assert_images_close, divergent, t32,
                     t64)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _scenes():
    a = synth.config(1, n_paths=1 << 13)
    b = synth.small_scene(n=16, n_cams=5, px=24, peak=25.0, seed=3, n_paths=1 << 12)
    c = synth.config(2, n_paths=1 << 11)
    c = c.replace(cameras=synth.arc_cameras(7, c.box_size, 40, 40))
    return [a, b, c]


def _oracle_parity(sc, scene_id, scene, paths_fp, beta_ref, beta_t, dldi, img, grad):
    """Oracle images / gradient for one scene, with the paths whose discrete
    decisions differ removed from both sides (same scheme as the per-scene
    parity tests)."""
    n = sc.n_paths
    ref = O.render(sc, beta_ref, beta_t, n=n, fingerprints=True, dldi=dldi, grad_abs=True, grad_cond=True,
                   image_cond=True, scene_id=scene_id)
    div = divergent(paths_fp, ref["fingerprints"])
    assert len(div) <= max(3, MAX_DIVERGENT * n)
    gi, gg = img.clone(), grad.clone()
    oi, og = ref["images"].copy(), ref["grad"].copy()
    for p in div:
        one = N.Paths(scene).store(t32(beta_ref), 1, sc.seed, first=int(p), n_norm=n)
        gi -= one.reweight(t32(beta_t))
        gg -= one.grad(t32(beta_t), t64(dldi))
        r1 = O.render(sc, beta_ref, beta_t, first=int(p), n=1, n_norm=n, dldi=dldi, scene_id=scene_id)
        oi -= r1["images"]
        og -= r1["grad"]
        one.close()
    torch.cuda.synchronize()
    return gi.cpu().numpy(), oi, gg.cpu().numpy(), og, ref["grad_abs"], ref["grad_cond"], ref["image_cond"]


def test_batch_matches_oracle_and_per_scene_calls():
    specs = _scenes()
    rng = np.random.default_rng(8)
    scenes = [N.Scene(sc, scene_id=i) for i, sc in enumerate(specs)]
    br = [sc.beta_cloud.astype(np.float32) for sc in specs]
    bt = [(sc.beta_cloud * rng.uniform(0.9, 1.15, size=sc.beta_cloud.shape)).astype(np.float32) for sc in specs]
    dl = [rng.standard_normal(s.n_pixels) for s in scenes]
    fps = [torch.zeros(sc.n_paths, dtype=torch.int64, device="cuda") for sc in specs]
    paths = [N.Paths(s).store(t32(b), sc.n_paths, sc.seed, fingerprints=f)
             for s, b, sc, f in zip(scenes, br, specs, fps)]
    # per-scene calls on the same stored paths
    btd = [t32(b) for b in bt]
    ref_img = [p.reweight(b, cache=True) for p, b in zip(paths, btd)]
    ref_grad = [p.grad(b, t64(d), cache=True) for p, b, d in zip(paths, btd, dl)]
    # one batched launch per pass over all three scenes
    imgs = [s.new_images() for s in scenes]
    grads = [torch.zeros(s.n_voxels, dtype=torch.float64, device="cuda") for s in scenes]
    batch = N.Batch(paths)
    batch.bind([t32(b) for b in bt], imgs, [t64(d) for d in dl], grads)
    batch.reweight(cache=True)
    batch.grad(cache=True)
    torch.cuda.synchronize()
    for s in scenes:
        s.check()
    first_img = [a.clone() for a in imgs]
    for k, sc in enumerate(specs):
        gi, oi, gg, og, oabs, ocond, icond = _oracle_parity(sc, k, scenes[k], fps[k], br[k], bt[k], dl[k], imgs[k], grads[k])
        assert np.abs(oi).max() > 0 and np.abs(og).max() > 0
        assert_images_close(gi, oi, what=f"batch images, scene {k}", cond=icond)
        assert_grad_close(gg, og, oabs, ocond, what=f"batch grad, scene {k}")
        # the batched and the per-scene kernels inline the same tile bodies
        # into different kernels; the compiler may contract a product into a
        # different FMA, so single contributions can differ by an FP32
        # rounding (about 1.2e-7 relative), never more
        assert_images_close(imgs[k].cpu().numpy(), ref_img[k].cpu().numpy(), rtol=1e-6,
                            what=f"batch vs per-scene images, scene {k}")
        assert_grad_close(grads[k].cpu().numpy(), ref_grad[k].cpu().numpy(), oabs, rtol=1e-6,
                          what=f"batch vs per-scene grad, scene {k}")
    # per-scene sequence (-1), grouped (0) and persistent schedules, both register variants
    cands = [(0, -1), (0, 1), (0, 4), (0, 0), (1, 0), (1, 2), (1, batch.launch_limit(1))]
    best, _ = tune_blocks(batch, scenes, [sc.n_paths for sc in specs], candidates=cands, reps=1,
                          use_cache=False)
    assert best in cands
    assert batch.launch_limit(1) >= batch.launch_limit(0)
    # every shape: the same contributions, only the order of the FP64 pixel
    # additions changes (the register-capped variant is another compilation
    # of the same bodies, so it is held to the FP32 rounding bound above)
    for shape in cands:
        batch.set_launch(*shape)
        batch.reweight(cache=True)
        torch.cuda.synchronize()
        for a, b in zip(imgs, first_img):
            if shape[0] == 0 and shape[1] >= 1:
                assert torch.allclose(a, b, rtol=1e-12, atol=0)
            else:
                assert_images_close(a.cpu().numpy(), b.cpu().numpy(), rtol=1e-6, what=f"shape {shape}")


def test_graph_replay_matches_eager_steps():
    specs = _scenes()
    def run(use_graph):
        scenes = [N.Scene(sc, scene_id=i) for i, sc in enumerate(specs)]
        gts = [0.7 * s.render_forward(t32(sc.beta_cloud), sc.n_paths, sc.seed + 3) for s, sc in zip(scenes, specs)]
        b0 = [torch.full((s.n_voxels,), float(sc.beta_cloud.mean()), dtype=torch.float32, device="cuda")
              for s, sc in zip(scenes, specs)]
        rec = BatchReconstruction(scenes, gts, b0, [sc.n_paths for sc in specs], n_r=3,
                                  lrs=[0.5] * len(specs))
        for _ in range(5):     # crosses a resample (t = 3)
            rec.step(use_graph=use_graph)
        torch.cuda.synchronize()
        return [b.cpu().numpy() for b in rec.beta], [l.item() for l in rec.loss]
    be, le = run(False)
    bg, lg = run(True)
    for a, b in zip(be, bg):
        assert np.allclose(a, b, rtol=1e-4, atol=1e-5)
    assert np.allclose(le, lg, rtol=1e-6)


def test_restore_repeats_steps_on_any_schedule():
    """A snapshot at a resample boundary, restored, repeats the same steps:
    three steps of the batched graph and three steps of per-scene calls from
    the same snapshot reach the same extinction and loss."""
    specs = _scenes()
    scenes = [N.Scene(sc, scene_id=i) for i, sc in enumerate(specs)]
    gts = [0.7 * s.render_forward(t32(sc.beta_cloud), sc.n_paths, sc.seed + 3) for s, sc in zip(scenes, specs)]
    b0 = [torch.full((s.n_voxels,), float(sc.beta_cloud.mean()), dtype=torch.float32, device="cuda")
          for s, sc in zip(scenes, specs)]
    rec = BatchReconstruction(scenes, gts, b0, [sc.n_paths for sc in specs], n_r=3, lrs=[0.5] * len(specs))
    for _ in range(3):
        rec.step(use_graph=True)
    assert rec.t % 3 == 0
    snap = rec.snapshot()
    rec.set_launch(1, 0)     # grouped, register-capped
    for _ in range(3):
        rec.step(use_graph=True)
    torch.cuda.synchronize()
    ba, la = [b.cpu().numpy() for b in rec.beta], [l.item() for l in rec.loss]
    rec.restore(snap)
    for _ in range(3):
        rec.step(batched=False)
    torch.cuda.synchronize()
    bb, lb = [b.cpu().numpy() for b in rec.beta], [l.item() for l in rec.loss]
    assert not all(np.array_equal(x, y.cpu().numpy()) for x, y in zip(ba, snap["beta"]))
    for a, b in zip(ba, bb):
        assert np.allclose(a, b, rtol=1e-4, atol=1e-5)
    assert np.allclose(la, lb, rtol=1e-6)
