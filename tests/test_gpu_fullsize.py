"""Parity at the full size of the timed workload (noise128: 128^3 grid, 15
cameras of 128x128, 2^24 paths), in the launch configuration the bench
times: one paths_store of all 2^24 paths, paths_reweight with the
contribution cache and render_grad from the cache.

No oracle run covers 2^24 paths, so the full launch is checked on outputs
the oracle computes path by path and on properties that hold at any size:
- fingerprints of sampled path ids (up to the last one) equal the oracle's;
- single-path stores of sampled ids, with the full run's normalisation,
  give the oracle's images and gradient element by element;
- the full launch equals the sum of two half launches (images to FP64
  summation order, gradient to the FP32 pre-sums of the merged reds);
- reweighting at beta_ref reproduces the store's own images, the tallies
  balance energy, and the path buckets and events match the tallies.
The batched workload (16 uneven scenes) is checked at its full size too:
every launch shape against the per-scene calls, and sampled fingerprints of
every scene against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2110_00085_gb300 import native as N
from paper_2110_00085_gb300 import synth

from _parity import assert_grad_close, assert_images_close, t32, t64

pytestmark = pytest.mark.gpu

FULL = 1 << 24


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def case():
    sc = synth.config(3, n_paths=FULL)
    rng = np.random.default_rng(24)
    br = sc.beta_cloud.astype(np.float32)
    bt = (sc.beta_cloud * rng.uniform(0.9, 1.15, size=sc.beta_cloud.shape)).astype(np.float32)
    scene = N.Scene(sc)
    dl = rng.standard_normal(scene.n_pixels)
    return sc, scene, br, bt, dl


@pytest.fixture(scope="module")
def full_run(case):
    sc, scene, br, bt, dl = case
    fp = torch.zeros(FULL, dtype=torch.int64, device="cuda")
    tal = torch.zeros(N.TALLY_COUNT, dtype=torch.float64, device="cuda")
    ref = scene.new_images()
    p = N.Paths(scene).store(t32(br), FULL, sc.seed, images_ref=ref, tallies=tal, fingerprints=fp)
    same = p.reweight(t32(br), cache=False)
    btd = t32(bt)
    img = p.reweight(btd, cache=True)
    g = p.grad(btd, t64(dl), cache=True)
    torch.cuda.synchronize()
    scene.check()
    out = {"fp": fp.cpu().numpy().view(np.uint64), "tallies": dict(zip(N.TALLY_NAMES, tal.cpu().numpy())),
           "ref": ref.cpu().numpy(), "same": same.cpu().numpy(), "img": img.cpu().numpy(),
           "grad": g.cpu().numpy(), "info": p.info()}
    p.close()
    return out


def test_fullsize_fingerprints_match_oracle_on_sampled_paths(case, full_run):
    sc, scene, br, bt, dl = case
    rng = np.random.default_rng(5)
    ids = np.unique(np.concatenate([rng.integers(0, FULL, 254), [0, FULL - 1]]))
    bad = 0
    for pid in ids:
        o = O.render(sc, br, first=int(pid), n=1, n_norm=FULL, fingerprints=True)["fingerprints"][0]
        bad += int(o != full_run["fp"][pid])
    assert bad <= 2, f"{bad} of {len(ids)} sampled paths take other discrete decisions"


def test_fullsize_sampled_paths_match_oracle_elementwise(case, full_run):
    """Path ids from the whole range, each stored alone with the full run's
    normalisation, summed on both sides and compared element by element."""
    sc, scene, br, bt, dl = case
    rng = np.random.default_rng(6)
    ids = [int(i) for i in rng.integers(0, FULL, 24)] + [FULL - 1]
    gi = scene.new_images()
    gg = torch.zeros(scene.n_voxels, dtype=torch.float64, device="cuda")
    oi = np.zeros(scene.n_pixels)
    og = np.zeros(scene.n_voxels)
    oabs = np.zeros(scene.n_voxels)
    ocond = np.zeros(scene.n_voxels)
    icond = np.zeros(scene.n_pixels)
    used = 0
    btd, dld = t32(bt), t64(dl)
    for pid in ids:
        o = O.render(sc, br, bt, first=pid, n=1, n_norm=FULL, dldi=dl, grad_abs=True, grad_cond=True,
                     image_cond=True, fingerprints=True)
        if o["fingerprints"][0] != full_run["fp"][pid]:
            continue    # a near-tie of a discrete decision: compared by neither side
        one = N.Paths(scene).store(t32(br), 1, sc.seed, first=pid, n_norm=FULL)
        one.reweight(btd, gi, cache=True, accumulate=True)
        one.grad(btd, dld, gg, cache=True, accumulate=True)
        one.close()
        oi += o["images"]; og += o["grad"]; oabs += o["grad_abs"]; ocond += o["grad_cond"]
        icond += o["image_cond"]
        used += 1
    torch.cuda.synchronize()
    assert used >= len(ids) - 2
    assert np.abs(oi).max() > 0 and np.abs(og).max() > 0
    assert_images_close(gi.cpu().numpy(), oi, cond=icond, what="sampled paths, images")
    # a few single paths: each touched voxel is crossed by one or two rays, so a
    # larger share of them rests on the float32 budget (measured 4.2%)
    assert_grad_close(gg.cpu().numpy(), og, oabs, ocond, what="sampled paths, gradient", max_budget_only=0.1)


def test_fullsize_launch_equals_two_half_launches(case, full_run):
    sc, scene, br, bt, dl = case
    half = FULL // 2
    img = scene.new_images()
    g = torch.zeros(scene.n_voxels, dtype=torch.float64, device="cuda")
    btd, dld = t32(bt), t64(dl)
    for first in (0, half):
        p = N.Paths(scene).store(t32(br), half, sc.seed, first=first, n_norm=FULL)
        p.reweight(btd, img, cache=True, accumulate=True)
        p.grad(btd, dld, g, cache=True, accumulate=True)
        torch.cuda.synchronize()
        p.close()
    scene.check()
    full_img, full_g = full_run["img"], full_run["grad"]
    assert np.abs(full_img).max() > 0
    assert_images_close(img.cpu().numpy(), full_img, rtol=1e-9, what="half + half vs full, images")
    g = g.cpu().numpy()
    scale = np.abs(full_g).max()
    # the merged reds pre-sum up to 8 FP32 terms, grouped differently in the
    # three launches: relative 1e-6 of the field, and 1e-5 per voxel on all
    # but a few voxels where the terms cancel
    assert np.linalg.norm(g - full_g) <= 1e-6 * np.linalg.norm(full_g)
    off = np.abs(g - full_g) > 1e-5 * np.abs(full_g) + 1e-9 * scale
    assert off.mean() < 1e-3, f"{off.sum()} voxels off"


def test_fullsize_invariants(full_run):
    # r == 1 at beta_ref: the store's own images, up to FP64 summation order
    assert np.abs(full_run["ref"]).max() > 0
    assert np.allclose(full_run["same"], full_run["ref"], rtol=1e-11, atol=0)
    T = full_run["tallies"]
    lhs = T["injected"] + T["rr_gain"]
    rhs = T["escaped"] + T["absorbed"] + T["truncated"] + T["rr_killed"]
    assert abs(lhs - rhs) < 1e-5 * lhs
    info = full_run["info"]
    bk = info["bucket"]
    w0 = T["injected"] / T["entered"]     # paths that miss the box hold no collisions
    assert sum(bk) == FULL and int(T["entered"]) + round(T["missed"] / w0) == FULL
    assert sum(k * c for k, c in enumerate(bk)) == int(T["collisions"])
    assert info["n_records"] == sum((k + 1) * c for k, c in enumerate(bk) if k >= 1)


def test_batch_fullsize_matches_per_scene_calls_and_oracle_fingerprints():
    """The batched workload at its full size (16 scenes of grid sides 32-128,
    5-21 cameras of 64x64, 2^20-2^23 paths each): the batched launches under
    the default and the grouped register-capped shapes agree with the
    per-scene calls on every scene, and sampled paths of every scene take
    the oracle's discrete decisions (scene id in the Philox counter)."""
    specs = synth.batch_config(5)
    rng = np.random.default_rng(44)
    scenes = [N.Scene(sc, scene_id=i) for i, sc in enumerate(specs)]
    br = [sc.beta_cloud.astype(np.float32) for sc in specs]
    bt = [(sc.beta_cloud * rng.uniform(0.9, 1.15, size=sc.beta_cloud.shape)).astype(np.float32) for sc in specs]
    dl = [rng.standard_normal(s.n_pixels) for s in scenes]
    fps, paths, ref_img, ref_g = [], [], [], []
    for s, sc, b, bb, d in zip(scenes, specs, br, bt, dl):
        fp = torch.zeros(sc.n_paths, dtype=torch.int64, device="cuda")
        p = N.Paths(s).store(t32(b), sc.n_paths, sc.seed, fingerprints=fp)
        bbd = t32(bb)
        ref_img.append(p.reweight(bbd, cache=True).cpu().numpy())
        ref_g.append(p.grad(bbd, t64(d), cache=True).cpu().numpy())
        fps.append(fp.cpu().numpy().view(np.uint64))
        paths.append(p)
    imgs = [s.new_images() for s in scenes]
    grads = [torch.zeros(s.n_voxels, dtype=torch.float64, device="cuda") for s in scenes]
    batch = N.Batch(paths)
    batch.bind([t32(b) for b in bt], imgs, [t64(d) for d in dl], grads)
    for shape in (batch.shape, (1, 0)):
        batch.set_launch(*shape)
        batch.reweight(cache=True)
        batch.grad(cache=True)
        torch.cuda.synchronize()
        for k, s in enumerate(scenes):
            s.check()
            assert np.abs(ref_img[k]).max() > 0
            assert_images_close(imgs[k].cpu().numpy(), ref_img[k], rtol=1e-6, what=f"shape {shape} scene {k}")
            g = grads[k].cpu().numpy()
            assert np.linalg.norm(g - ref_g[k]) <= 1e-6 * np.linalg.norm(ref_g[k])
    batch.close()
    for p in paths:
        p.close()
    bad = 0
    for k, sc in enumerate(specs):
        for pid in rng.integers(0, sc.n_paths, 4):
            o = O.render(sc, br[k], first=int(pid), n=1, n_norm=sc.n_paths, fingerprints=True, scene_id=k)
            bad += int(o["fingerprints"][0] != fps[k][pid])
    assert bad <= 1


def test_cumulus256_chunked_fullsize():
    """The large reconstruction at full size (256^3 fractal cumulus in air,
    21 cameras of 256x256, 2^28 paths), stored as four chunks of 2^26 path
    ids: fingerprints of sampled ids across all chunks and single-path
    stores match the oracle; reweighting at beta_ref gives the store's own
    images; the tallies balance energy and match the buckets."""
    from paper_2110_00085_gb300.driver import ChunkedPaths
    n = 1 << 28
    sc = synth.config(5, n_paths=n)
    scene = N.Scene(sc)
    rng = np.random.default_rng(55)
    br = sc.beta_cloud.astype(np.float32)
    bt = (sc.beta_cloud * rng.uniform(0.9, 1.15, size=sc.beta_cloud.shape)).astype(np.float32)
    dl = rng.standard_normal(scene.n_pixels)
    cp = ChunkedPaths(scene)
    fp = torch.zeros(n, dtype=torch.int64, device="cuda")
    tal = torch.zeros(N.TALLY_COUNT, dtype=torch.float64, device="cuda")
    ref = scene.new_images()
    cp.store(t32(br), n, sc.seed, images_ref=ref, tallies=tal, fingerprints=fp)
    assert len(cp.parts) == 4
    same = cp.reweight(t32(br), cache=False)
    btd = t32(bt)
    img = cp.reweight(btd, cache=True)
    g = cp.grad(btd, t64(dl), cache=True)
    torch.cuda.synchronize()
    scene.check()
    info = cp.info()
    cp.close()
    assert np.abs(img.cpu().numpy()).max() > 0 and np.abs(g.cpu().numpy()).max() > 0
    assert torch.allclose(same, ref, rtol=1e-11, atol=0)
    T = dict(zip(N.TALLY_NAMES, tal.cpu().numpy()))
    assert abs(T["injected"] + T["rr_gain"] - T["escaped"] - T["absorbed"] - T["truncated"] - T["rr_killed"]) \
        < 1e-5 * T["injected"]
    # every path has a bucket (paths that miss the box hold no collisions)
    bk = info["bucket"]
    w0 = T["injected"] / T["entered"]
    assert sum(bk) == n and int(T["entered"]) + round(T["missed"] / w0) == n
    assert sum(k * c for k, c in enumerate(bk)) == int(T["collisions"])
    fph = fp.cpu().numpy().view(np.uint64)
    del fp
    ids = [int(i) for i in rng.integers(0, n, 60)] + [0, (1 << 26) - 1, 1 << 26, n - 1]
    bad = sum(int(O.render(sc, br, first=pid, n=1, n_norm=n, fingerprints=True)["fingerprints"][0] != fph[pid])
              for pid in ids)
    assert bad <= 1
    # single-path stores of sampled ids against the oracle, element by element
    gi = scene.new_images()
    gg = torch.zeros(scene.n_voxels, dtype=torch.float64, device="cuda")
    oi = np.zeros(scene.n_pixels); icond = np.zeros(scene.n_pixels)
    og = np.zeros(scene.n_voxels); oabs = np.zeros(scene.n_voxels); ocond = np.zeros(scene.n_voxels)
    used = 0
    dld = t64(dl)
    for pid in ids[:12] + [n - 1]:
        o = O.render(sc, br, bt, first=pid, n=1, n_norm=n, dldi=dl, grad_abs=True, grad_cond=True,
                     image_cond=True, fingerprints=True)
        if o["fingerprints"][0] != fph[pid]:
            continue
        one = N.Paths(scene).store(t32(br), 1, sc.seed, first=pid, n_norm=n)
        one.reweight(btd, gi, cache=True, accumulate=True)
        one.grad(btd, dld, gg, cache=True, accumulate=True)
        one.close()
        oi += o["images"]; icond += o["image_cond"]
        og += o["grad"]; oabs += o["grad_abs"]; ocond += o["grad_cond"]
        used += 1
    torch.cuda.synchronize()
    assert used >= 11 and np.abs(oi).max() > 0
    assert_images_close(gi.cpu().numpy(), oi, cond=icond, what="cumulus256 sampled paths, images")
    # thirteen single paths through 256^3 voxels with 21 cameras: each touched
    # voxel is crossed by one ray or two; 21% of them rest on the float32
    # budget (1.2% of the gradient's term mass), measured
    assert_grad_close(gg.cpu().numpy(), og, oabs, ocond, what="cumulus256 sampled paths, gradient",
                      max_budget_only=0.3)
