"""CUDA path vs. the FP64 oracle, element by element, on identical Philox
streams (relative 1e-4 per pixel and per voxel), plus the invariants that
hold at any size.  Needs a GB300."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2110_00085_gb300 import native as N
from paper_2110_00085_gb300 import synth

from _parity import (RTOL, THREADS, assert_grad_close, assert_images_close, forward_parity, recycled_parity, t32,
                     t64)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _perturbed(beta, seed=0, lo=0.85, hi=1.2):
    rng = np.random.default_rng(seed)
    return (beta * rng.uniform(lo, hi, size=beta.shape)).astype(np.float32)


# ------------------------------------------------------------ forward ------
@pytest.mark.parametrize("cfg,n,first", [(1, 1 << 14, 0), (1, 5000, 123457), (2, 1 << 11, 0)])
def test_forward_matches_oracle(cfg, n, first):
    """Plain path tracing (Alg. 1 forward): 2^14 paths (many tiles) and a
    ragged count at an offset path id; workload 2 has air (two types)."""
    sc = synth.config(cfg, n_paths=n)
    gi, oi, tg, to, nd, ic = forward_parity(sc, sc.beta_cloud, n, first=first)
    assert np.abs(oi).max() > 0
    assert_images_close(gi, oi, cond=ic)
    # tallies: collision and path counts are integers; weights FP32-summed
    names = N.TALLY_NAMES
    for k in ("entered", "collisions"):
        assert abs(tg[names.index(k)] - to[k]) <= 2 * nd + 1
    for k in ("injected", "escaped", "absorbed"):
        assert abs(tg[names.index(k)] - to[k]) <= 1e-3 * to["injected"]


def test_energy_balance_on_gpu():
    sc = synth.config(1, n_paths=1 << 16)
    scene = N.Scene(sc)
    tal = torch.zeros(N.TALLY_COUNT, dtype=torch.float64, device="cuda")
    scene.render_forward(t32(sc.beta_cloud), sc.n_paths, sc.seed, tallies=tal)
    T = dict(zip(N.TALLY_NAMES, tal.cpu().numpy()))
    lhs = T["injected"] + T["rr_gain"]
    rhs = T["escaped"] + T["absorbed"] + T["truncated"] + T["rr_killed"]
    assert abs(lhs - rhs) < 1e-5 * lhs


def test_forward_chunks_add_up():
    """Two calls over disjoint path ranges accumulate to the one-call image."""
    sc = synth.config(1, n_paths=1 << 13)
    scene = N.Scene(sc)
    b = t32(sc.beta_cloud)
    n = sc.n_paths
    full = scene.render_forward(b, n, sc.seed)
    part = scene.render_forward(b, 3000, sc.seed, n_norm=n)
    scene.render_forward(b, n - 3000, sc.seed, first=3000, n_norm=n, images=part, accumulate=True)
    assert torch.allclose(full, part, rtol=1e-12, atol=0)


# ------------------------------------------------------------ recycling ---
@pytest.mark.parametrize("cfg,n", [(1, 1 << 14), (2, 1 << 11)])
def test_recycled_forward_matches_oracle(cfg, n):
    """Paths stored under M_ref, reweighted to M_t (Eq. 19/20)."""
    sc = synth.config(cfg, n_paths=n)
    bt = _perturbed(sc.beta_cloud, seed=cfg)
    out = recycled_parity(sc, sc.beta_cloud, bt, n)
    assert_images_close(out["gpu_images"], out["oracle_images"], what="recycled images",
                        cond=out["oracle_image_cond"])


def test_recycling_ratio_is_one_at_reference():
    """r == 1 when M_t == M_ref: the recycled pass reproduces the store's own
    plain estimate (same contributions, only the FP64 summation order differs)."""
    sc = synth.config(1, n_paths=1 << 15)
    scene = N.Scene(sc)
    b = t32(sc.beta_cloud)
    ref = scene.new_images()
    paths = N.Paths(scene).store(b, sc.n_paths, sc.seed, images_ref=ref)
    again = paths.reweight(b.clone())
    plain = scene.render_forward(b, sc.n_paths, sc.seed)
    assert torch.allclose(again, ref, rtol=1e-11, atol=0)
    assert torch.allclose(plain, ref, rtol=1e-11, atol=0)


def test_sorted_buckets_are_consistent():
    """Counting sort: bucket sizes add up to the stored paths, and sum B*count
    equals the collision tally."""
    sc = synth.config(1, n_paths=1 << 15)
    scene = N.Scene(sc)
    b = t32(sc.beta_cloud)
    tal = torch.zeros(N.TALLY_COUNT, dtype=torch.float64, device="cuda")
    paths = N.Paths(scene).store(b, sc.n_paths, sc.seed, tallies=tal)
    info = paths.info()
    T = dict(zip(N.TALLY_NAMES, tal.cpu().numpy()))
    bk = info["bucket"]
    assert sum(bk[1:]) == info["n_stored"]
    assert sum(k * c for k, c in enumerate(bk)) == int(T["collisions"])
    assert sum(bk) == int(T["entered"])
    assert info["n_records"] == sum((k + 1) * c for k, c in enumerate(bk) if k >= 1)


# ------------------------------------------------------------ gradient -----
@pytest.mark.parametrize("cfg,n,cache", [(1, 1 << 13, False), (1, 1 << 13, True), (2, 1 << 10, True)])
def test_gradient_matches_oracle(cfg, n, cache):
    """render_grad (Eq. 21 with the PSF of Sec. 4.4) vs. the oracle's
    term-by-term gradient, per voxel, relative to the voxel's term mass."""
    sc = synth.config(cfg, n_paths=n)
    bt = _perturbed(sc.beta_cloud, seed=10 + cfg)
    gt = 0.8 * O.render(sc, sc.beta_cloud, n=n, seed=sc.seed + 99)["images"]
    F = O.render(sc, sc.beta_cloud, bt, n=n)["images"]
    dldi = F - gt
    out = recycled_parity(sc, sc.beta_cloud, bt, n, dldi=dldi, cache=cache)
    assert np.abs(out["oracle_grad"]).max() > 0
    assert_grad_close(out["gpu_grad"], out["oracle_grad"], out["oracle_grad_abs"], out["oracle_grad_cond"])


def test_noise128_consecutive_paths_match_oracle_elementwise():
    """The timed workload's grid and cameras (128^3 thresholded noise, 15
    cameras of 128x128): one store of 2^14 consecutive paths, cached
    reweight and cached gradient as in the timed step, compared element by
    element -- the gradient kernel's warps sum same-voxel terms of different
    paths' events (lateral ray order, run merge) before their FP64 adds."""
    n = 1 << 14
    sc = synth.config(3, n_paths=n)
    bt = _perturbed(sc.beta_cloud, seed=33, lo=0.9, hi=1.1)
    gt = 0.8 * O.render(sc, sc.beta_cloud, n=n, seed=sc.seed + 99, threads=THREADS)["images"]
    F = O.render(sc, sc.beta_cloud, bt, n=n, threads=THREADS)["images"]
    out = recycled_parity(sc, sc.beta_cloud, bt, n, dldi=F - gt, cache=True)
    assert np.abs(out["oracle_images"]).max() > 0 and np.abs(out["oracle_grad"]).max() > 0
    assert_images_close(out["gpu_images"], out["oracle_images"], what="noise128 images",
                        cond=out["oracle_image_cond"])
    assert_grad_close(out["gpu_grad"], out["oracle_grad"], out["oracle_grad_abs"], out["oracle_grad_cond"],
                      what="noise128 gradient")


def test_gradient_cache_equals_recompute():
    sc = synth.config(1, n_paths=1 << 14)
    scene = N.Scene(sc)
    br, bt = t32(sc.beta_cloud), t32(_perturbed(sc.beta_cloud, 5))
    paths = N.Paths(scene).store(br, sc.n_paths, sc.seed)
    img = paths.reweight(bt, cache=True)
    dldi = img - 0.5 * img.mean()
    g1 = paths.grad(bt, dldi, cache=True)
    g2 = paths.grad(bt, dldi, cache=False)
    # the event kernel pre-sums up to 8 same-voxel FP32 terms per warp step
    # before its FP64 red (a few units of roundoff of those terms)
    assert torch.allclose(g1, g2, rtol=1e-5, atol=1e-7 * g2.abs().max().item())


def test_gradient_cache_equals_recompute_dense_events():
    """Many events per voxel (tiny grid, many paths): warps hold long runs of
    same-voxel events, so the per-step merging of their shadow-ray terms is
    exercised across 8-lane chunk boundaries."""
    sc = synth.small_scene(n=6, n_cams=4, px=8, peak=30.0, seed=13, n_paths=1 << 16)
    scene = N.Scene(sc)
    br, bt = t32(sc.beta_cloud), t32(_perturbed(sc.beta_cloud, 6))
    paths = N.Paths(scene).store(br, sc.n_paths, sc.seed)
    img = paths.reweight(bt, cache=True)
    dldi = img - 0.4 * img.mean()
    g1 = paths.grad(bt, dldi, cache=True)
    g2 = paths.grad(bt, dldi, cache=False)
    assert g2.abs().max().item() > 0
    assert torch.allclose(g1, g2, rtol=1e-5, atol=1e-7 * g2.abs().max().item())


# ------------------------------------------------------------ edge cases ---
def test_empty_medium_gives_zero():
    sc = synth.config(1, n_paths=1 << 10)
    scene = N.Scene(sc)
    z = torch.zeros(sc.n_voxels, dtype=torch.float32, device="cuda")
    img = scene.render_forward(z, sc.n_paths, sc.seed)
    assert img.abs().max().item() == 0.0
    paths = N.Paths(scene).store(z, sc.n_paths, sc.seed)
    assert paths.info()["n_stored"] == 0
    assert paths.reweight(z).abs().max().item() == 0.0
    g = paths.grad(z, torch.ones(scene.n_pixels, dtype=torch.float64, device="cuda"))
    assert g.abs().max().item() == 0.0
    # the cached pass with no events at all (buffers sized from the counts)
    assert paths.reweight(z, cache=True).abs().max().item() == 0.0
    g = paths.grad(z, torch.ones(scene.n_pixels, dtype=torch.float64, device="cuda"), cache=True)
    assert g.abs().max().item() == 0.0
    # a handle reused for a larger path set grows its buffers
    paths.store(t32(sc.beta_cloud), sc.n_paths, sc.seed)
    img2 = paths.reweight(t32(sc.beta_cloud), cache=True)
    ref = scene.render_forward(t32(sc.beta_cloud), sc.n_paths, sc.seed)
    torch.cuda.synchronize()
    assert torch.allclose(img2, ref, rtol=1e-11, atol=0)


def test_single_path_and_first_order_only():
    sc = synth.config(1, n_paths=1).replace(max_orders=1)
    gi, oi, *_, ic = forward_parity(sc, sc.beta_cloud, 64, first=777)
    assert_images_close(gi, oi, cond=ic)


def test_invalid_arguments_raise():
    sc = synth.config(1, n_paths=16)
    scene = N.Scene(sc)
    with pytest.raises(ValueError):
        scene.render_forward(torch.zeros(5, device="cuda"), 16, 1)
    bad = sc.replace(max_orders=99)
    with pytest.raises(RuntimeError):
        N.Scene(bad)
    p = N.Paths(scene)
    with pytest.raises(RuntimeError):
        p.reweight(t32(sc.beta_cloud))


# ------------------------------------------------------------ loss, Adam ---
def test_loss_residual_and_adam_match_reference():
    rng = np.random.default_rng(3)
    img = rng.normal(size=1000)
    gt = rng.normal(size=1000)
    d, loss = N.loss_residual(t64(img), t64(gt))
    assert np.allclose(d.cpu().numpy(), img - gt, rtol=0, atol=0)
    assert abs(loss.item() - 0.5 * np.sum((img - gt) ** 2)) < 1e-12 * np.sum((img - gt) ** 2)
    beta = rng.uniform(0, 5, size=4096).astype(np.float32)
    g = rng.normal(size=4096) * 1e-3
    m = np.zeros(4096, np.float32)
    v = np.zeros(4096, np.float32)
    tb, tm, tv = t32(beta), t32(m), t32(v)
    rb, rm, rv = beta.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for t in range(1, 6):
        N.adam_step(tb, tm, tv, t64(g * t), t, lr=0.1)
        rb, rm, rv = O.adam_step(rb, rm, rv, g * t, t, lr=0.1)
    assert np.allclose(tb.cpu().numpy(), rb, rtol=1e-5, atol=1e-5)
    assert (tb.cpu().numpy() >= 0).all()


def test_device_error_word_is_reported_once_and_cleared():
    """The reporting path of kernel-side invariant checks: bits recorded in
    the scene's error word (here by the host hook, as a kernel would) make
    the next check raise with their meaning and are cleared by it."""
    sc = synth.config(1, n_paths=1 << 10)
    scene = N.Scene(sc)
    scene.check()
    scene.inject_error(2)
    with pytest.raises(RuntimeError, match="0x2"):
        scene.check()
    scene.check()
    scene.inject_error(1)
    scene.inject_error(4)
    with pytest.raises(RuntimeError, match="0x5"):
        scene.check()
    scene.check()


def test_store_rejects_invalid_extinction_before_tracing():
    """A grid with a NaN, an infinite or a negative voxel is refused with a
    status naming the count (no path kernel runs on it); the handle holds no
    paths afterwards and a valid store on it works."""
    sc = synth.config(1, n_paths=1 << 10)
    scene = N.Scene(sc)
    good = torch.from_numpy(sc.beta_cloud.reshape(-1).astype(np.float32)).cuda()
    for bad_value in (float("nan"), float("inf"), -1.0):
        b = good.clone()
        b[[5, 77]] = bad_value
        P = N.Paths(scene)
        with pytest.raises(RuntimeError, match="2 voxels"):
            P.store(b, 1 << 10, 1)
        with pytest.raises(RuntimeError, match="no paths"):
            P.reweight(good)
        P.store(good, 1 << 10, 1)
        assert float(P.reweight(good).sum()) > 0
        P.close()
    scene.check()


def test_async_store_equals_synchronous_store():
    """paths_store(PT_ASYNC) on a handle that a synchronous store has sized
    stores the same paths as a synchronous store (images and gradient equal
    to FP64 summation order) without synchronising."""
    sc = synth.config(1, n_paths=1 << 14)
    scene = N.Scene(sc)
    b = t32(sc.beta_cloud)
    bt = t32(_perturbed(sc.beta_cloud, 8))
    A = N.Paths(scene).store(b, sc.n_paths, sc.seed, epoch=0)
    A.store(b, sc.n_paths, sc.seed, epoch=1, asynchronous=True)
    ia = A.reweight(bt, cache=True)
    dl = ia - 0.5 * ia.mean()
    ga = A.grad(bt, dl, cache=True)
    B = N.Paths(scene).store(b, sc.n_paths, sc.seed, epoch=1)
    ib = B.reweight(bt, cache=True)
    gb = B.grad(bt, dl, cache=True)
    torch.cuda.synchronize()
    scene.check()
    assert float(ib.sum()) > 0
    assert torch.allclose(ia, ib, rtol=1e-12, atol=0)
    assert float((ga - gb).abs().sum()) <= 1e-9 * float(gb.abs().sum())
    assert A.info()["n_stored"] == B.info()["n_stored"]
    A.close()
    B.close()


def test_async_store_reports_what_it_cannot_hold():
    """A PT_ASYNC store of an invalid grid, or of more records than the
    handle's buffers hold, leaves the handle without paths (later passes add
    nothing) and is reported by pt_check (bit 8); a synchronous store then
    grows the buffers and works."""
    sc = synth.config(1, n_paths=1 << 10)
    scene = N.Scene(sc)
    good = t32(sc.beta_cloud)
    P = N.Paths(scene).store(good, 1 << 10, 1)
    bad = good.clone()
    bad[[3, 9]] = float("nan")
    P.store(bad, 1 << 10, 1, asynchronous=True)
    assert float(P.reweight(good).abs().sum()) == 0.0
    with pytest.raises(RuntimeError, match="0x8"):
        scene.check()
    P.store(good, 1 << 14, 2, asynchronous=True)   # about 16x the records the buffers hold
    assert float(P.reweight(good).abs().sum()) == 0.0
    assert P.info()["n_stored"] == 0
    with pytest.raises(RuntimeError, match="0x8"):
        scene.check()
    P.store(good, 1 << 14, 2)
    assert float(P.reweight(good).sum()) > 0
    scene.check()
    P.close()


def test_lean_chunked_cache_equals_full_cache():
    """A path set in four handles, keeping one handle's contribution cache at
    a time (reweight without the cache, then per handle reweight with it,
    gradient, drop): the same images and gradient as with every cache kept,
    and the caches are freed."""
    from paper_2110_00085_gb300.driver import ChunkedPaths
    sc = synth.config(1, n_paths=1 << 14)
    scene = N.Scene(sc)
    b = t32(sc.beta_cloud)
    bt = t32(_perturbed(sc.beta_cloud, 9))
    full = ChunkedPaths(scene, chunk=1 << 12).store(b, sc.n_paths, sc.seed)
    lean = ChunkedPaths(scene, chunk=1 << 12, lean=True).store(b, sc.n_paths, sc.seed)
    assert len(full.parts) == 4 and len(lean.parts) == 4
    i1 = full.reweight(bt, cache=True)
    dl = i1 - 0.5 * i1.mean()
    g1 = full.grad(bt, dl, cache=True)
    i2 = lean.reweight(bt, cache=True)
    g2 = lean.grad(bt, dl, cache=True)
    torch.cuda.synchronize()
    scene.check()
    assert torch.allclose(i1, i2, rtol=1e-12, atol=0)
    assert float((g1 - g2).abs().sum()) <= 1e-9 * float(g1.abs().sum())
    assert lean.info()["bytes_device"] < full.info()["bytes_device"]
    full.close()
    lean.close()


def test_repeated_passes_agree_to_summation_order():
    """Determinism: the same recycled forward and gradient run twice on the
    same stored paths agree to FP64 summation-order noise (the atomics'
    order is the only freedom), with and without the contribution cache."""
    sc = synth.config(1, n_paths=1 << 14)
    scene = N.Scene(sc)
    bt = torch.from_numpy(sc.beta_cloud.reshape(-1).astype(np.float32)).cuda()
    P = N.Paths(scene).store(bt, 1 << 14, 3)
    b1 = bt * 1.05
    for cache in (True, False):
        i1 = P.reweight(b1, cache=cache).clone()
        dl = i1 - 0.9 * i1.mean()
        g1 = P.grad(b1, dl, cache=cache).clone()
        i2 = P.reweight(b1, cache=cache)
        g2 = P.grad(b1, dl, cache=cache)
        torch.cuda.synchronize()
        assert torch.allclose(i1, i2, rtol=1e-12, atol=0)
        assert float((g1 - g2).abs().sum()) <= 1e-9 * float(g1.abs().sum())
    P.close()
