"""Helpers for comparing the CUDA path with the oracle on identical Philox
streams.

FP32 path arithmetic on the GPU and FP64 in the oracle take the same discrete
decisions (collision voxel, escape, roulette, particle type, pixel) except for
rare near-ties.  Both sides emit a per-path fingerprint of those decisions;
the paths whose fingerprints differ are rendered one by one on each side
(same path id, same normalisation) and removed from both totals before the
element-wise comparison.  No value computed by the CUDA path enters the
oracle: only the list of path ids to leave out is shared.
"""
import os

import numpy as np
import torch

import oracle as O
from paper_2110_00085_gb300 import native as N

RTOL = 1e-4          # per pixel, per voxel (of the voxel's absolute term mass)
MAX_DIVERGENT = 2e-3  # fraction of paths whose discrete decisions may differ
U32 = 2.0 ** -24      # FP32 unit roundoff
THREADS = os.cpu_count() or 1   # oracle threads (the split does not change its results)
# Elements (lit pixels, touched voxels) that pass only through the oracle's
# measured float32 budget -- their error exceeds RTOL of the value (pixels)
# or of the term mass (voxels) -- may be at most this fraction of the
# non-zero elements; every comparison prints its count and the largest
# budget / (RTOL x value) ratio, and their share of the summed magnitude
# (|value| or term mass).  Small path sets need the budget most: a voxel
# crossed by few rays, one of them ill-conditioned.
MAX_BUDGET_ONLY = 5e-2
MAX_BUDGET_SHARE = 2e-2   # ... and their share of the summed magnitude


def t32(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.float32).reshape(-1))).cuda()


def t64(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.float64).reshape(-1))).cuda()


def divergent(fp_gpu: torch.Tensor, fp_oracle: np.ndarray, first: int = 0):
    g = fp_gpu.cpu().numpy().view(np.uint64)
    return np.nonzero(g != fp_oracle)[0] + first


def assert_images_close(gi, oi, rtol=RTOL, what="images", cond=None, max_budget_only=MAX_BUDGET_ONLY,
                        max_budget_share=MAX_BUDGET_SHARE):
    """Per pixel: |gpu - oracle| <= rtol |oracle| + cond, where cond (the
    oracle's image_cond) is the measured float32 sensitivity of the pixel's
    contributions: large only where a path's geometry is ill-conditioned (a
    collision in thin air just past cloud edges, a near-tie of the pixel)."""
    gi = np.asarray(gi)
    oi = np.asarray(oi)
    floor = 1e-9 * max(np.abs(oi).max(), 1e-300)
    atol = floor
    if cond is not None:
        atol = atol + np.asarray(cond)
    err = np.abs(gi - oi)
    bad = err > rtol * np.abs(oi) + atol
    if bad.any():
        budget = rtol * np.abs(oi) + atol
        k = np.argmax(err / budget)
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} elements off; worst at {k}: "
                             f"gpu {gi[k]:.9e} oracle {oi[k]:.9e} budget {np.broadcast_to(budget, oi.shape)[k]:.3e}")
    _budget_report(what, err, rtol * np.abs(oi) + floor, cond, oi != 0, np.abs(oi), max_budget_only,
                   max_budget_share)


def assert_grad_close(gg, og, oabs, ocond=None, rtol=RTOL, what="grad", max_budget_only=MAX_BUDGET_ONLY,
                      max_budget_share=MAX_BUDGET_SHARE):
    """Per voxel: |g_gpu - g_oracle| <= rtol * sum|terms| + cond, where
    cond (the oracle's grad_cond) is the measured float32 sensitivity of the
    voxel's gradient terms (the change under perturbed re-sampling of the
    paths, plus the roundoff of the crossing times)."""
    gg = np.asarray(gg)
    err = np.abs(gg - og)
    floor0 = 1e-12 * max(oabs.max(), 1e-300)
    floor = floor0
    if ocond is not None:
        floor = floor + ocond
    bad = err > rtol * oabs + floor
    if bad.any():
        budget = rtol * oabs + floor
        k = np.argmax(err / budget)
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} voxels off; worst at {k}: gpu {gg[k]:.9e} "
                             f"oracle {og[k]:.9e} |terms| {oabs[k]:.3e} budget {budget[k]:.3e}")
    _budget_report(what, err, rtol * oabs + floor0, ocond, oabs != 0, oabs, max_budget_only, max_budget_share)


def _budget_report(what, err, base, cond, nonzero, mag, max_budget_only, max_budget_share):
    """Counts the elements whose error exceeds the base tolerance (RTOL of
    the value or term mass) and that pass only through the float32 budget;
    prints the count, their share of the summed magnitude and the largest
    budget / base ratio, and bounds the count by max_budget_only of the
    non-zero elements and the share by max_budget_share."""
    n = int(np.count_nonzero(nonzero))
    over = (err > base) & nonzero
    k = int(np.count_nonzero(over))
    ratio = 0.0
    if cond is not None and n:
        c = np.broadcast_to(np.asarray(cond, dtype=np.float64), err.shape)[nonzero]
        ratio = float(np.max(c / np.maximum(base[nonzero], 1e-300)))
    share = float(mag[over].sum()) / max(float(mag.sum()), 1e-300)
    print(f"[parity] {what}: {k} of {n} non-zero elements pass only through the float32 budget "
          f"({k / max(n, 1):.2e}, {share:.2e} of the magnitude); largest budget / ({RTOL:g} x value) = {ratio:.3g}")
    assert k <= max_budget_only * n, (f"{what}: {k} of {n} non-zero elements need the float32 budget "
                                      f"(more than {max_budget_only:g})")
    assert share <= max_budget_share, (f"{what}: elements that need the float32 budget carry {share:.3g} of the "
                                       f"magnitude (more than {max_budget_share:g})")


def forward_parity(sc, beta, n, first=0, seed=None):
    """Returns (gpu images, oracle images) with divergent paths removed."""
    seed = sc.seed if seed is None else seed
    scene = N.Scene(sc)
    b = t32(beta)
    fp = torch.zeros(n, dtype=torch.int64, device="cuda")
    tal = torch.zeros(N.TALLY_COUNT, dtype=torch.float64, device="cuda")
    img = scene.render_forward(b, n, seed, first=first, tallies=tal, fingerprints=fp)
    ref = O.render(sc, beta, first=first, n=n, seed=seed, fingerprints=True, tallies=True, image_cond=True,
                   threads=THREADS)
    div = divergent(fp, ref["fingerprints"], first)
    print(f"[parity] forward: {len(div)} of {n} paths divergent ({len(div) / n:.2e})")
    assert len(div) <= max(3, MAX_DIVERGENT * n), f"{len(div)} divergent paths of {n}"
    gi = img.clone()
    oi = ref["images"].copy()
    for p in div:
        e = scene.render_forward(b, 1, seed, first=int(p), n_norm=n)
        gi -= e
        oi -= O.render(sc, beta, first=int(p), n=1, n_norm=n, seed=seed)["images"]
    torch.cuda.synchronize()
    scene.check()
    return gi.cpu().numpy(), oi, tal.cpu().numpy(), ref["tallies"], len(div), ref["image_cond"]


def recycled_parity(sc, beta_ref, beta_t, n, dldi=None, cache=False, first=0):
    """Paths stored under beta_ref, evaluated under beta_t, on both sides.
    Returns dict of gpu/oracle images (and gradients), divergent removed."""
    scene = N.Scene(sc)
    br, bt = t32(beta_ref), t32(beta_t)
    fp = torch.zeros(n, dtype=torch.int64, device="cuda")
    paths = N.Paths(scene).store(br, n, sc.seed, first=first, fingerprints=fp)
    img = paths.reweight(bt, cache=cache)
    ref = O.render(sc, beta_ref, beta_t, first=first, n=n, fingerprints=True, image_cond=True,
                   dldi=dldi, grad_abs=dldi is not None, grad_cond=dldi is not None, threads=THREADS)
    out = {"gpu_images": img, "oracle_images": ref["images"].copy(), "oracle_image_cond": ref["image_cond"]}
    if dldi is not None:
        g = paths.grad(bt, t64(dldi), cache=cache)
        out["gpu_grad"] = g
        out["oracle_grad"] = ref["grad"].copy()
        out["oracle_grad_abs"] = ref["grad_abs"]
        out["oracle_grad_cond"] = ref["grad_cond"]
    div = divergent(fp, ref["fingerprints"], first)
    print(f"[parity] recycled: {len(div)} of {n} paths divergent ({len(div) / n:.2e})")
    assert len(div) <= max(3, MAX_DIVERGENT * n), f"{len(div)} divergent paths of {n}"
    for p in div:
        one = N.Paths(scene).store(br, 1, sc.seed, first=int(p), n_norm=n)
        out["gpu_images"] -= one.reweight(bt)
        r1 = O.render(sc, beta_ref, beta_t, first=int(p), n=1, n_norm=n, dldi=dldi)
        out["oracle_images"] -= r1["images"]
        if dldi is not None:
            out["gpu_grad"] -= one.grad(bt, t64(dldi))
            out["oracle_grad"] -= r1["grad"]
        one.close()
    torch.cuda.synchronize()
    scene.check()
    out["gpu_images"] = out["gpu_images"].cpu().numpy()
    if dldi is not None:
        out["gpu_grad"] = out["gpu_grad"].cpu().numpy()
    out["divergent"] = len(div)
    out["paths"] = paths
    out["scene"] = scene
    return out
