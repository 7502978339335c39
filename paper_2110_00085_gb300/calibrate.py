"""Gradient error of path reuse vs resampling, and the resample path budget
of equal error (Sec. 5: recycled paths trade variance for speed).

matched_errors measures both estimators against a reference gradient
g_ref (the mean of 16 fresh gradients of 4N paths each) as
||g - g_ref|| / ||g_ref||, in L2 and in L1, at extinctions of one recycling
window; the functions below it measure the spread of two independent
estimates instead (no reference needed):

Both estimators are unbiased up to the correlation of a gradient with the
images of the same paths, so their error is measured as their spread: the
difference of two estimates from independent path sets at the same
extinction, with no high-budget reference needed.  Errors are matched in
absolute terms at the same extinctions, in two norms:
- L1 (the matching norm): mean over voxels of |g_a - g_b|.  The local
  estimate toward a camera near the phase function's forward peak makes
  rare events with large terms, so squared errors are dominated by a few
  voxels (a single voxel often carries half of ||g_a - g_b||^2) and converge
  slowly; the mean absolute difference follows the n^(-1/2) law closely
  already at moderate budgets, and Adam, which divides each voxel's step by
  its running RMS, is itself insensitive to such single-voxel spikes.
- L2 (reported): sqrt(||g_a - g_b||^2 / 2), the standard error summed over
  voxels.
For reading, the signal norm ||g||^2 = E||(g_a + g_b)/2||^2 -
E||g_a - g_b||^2 / 4 (the noise part removed) is reported too; at small
budgets on large grids the per-voxel noise dominates and it is 0.

- Reuse (Alg. 2): paths stored at beta_ref serve N_r Adam steps; the error
  grows as beta_t moves away from beta_ref.  One recycling window is run
  with path set A (which drives the optimisation) while an independent set
  B, stored at the same beta_ref, is evaluated at every beta_t; e_reuse is
  the RMS over the window's steps.
- Resample (Alg. 1): fresh paths at beta_t every step.  Two fresh sets per
  beta_t and path budget n' give e_resample(n'); it falls as n'^(-1/2).
- n_star: the resample budget whose error equals e_reuse, from a line
  fitted to log e_resample against log n'.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence

import torch

from . import native as N


def grad_error(g_a: torch.Tensor, g_b: torch.Tensor) -> float:
    """L1 spread of two independent estimates of one gradient: the mean over
    voxels of |g_a - g_b|."""
    return float((g_a - g_b).double().abs().mean())


def grad_error_l2(g_a: torch.Tensor, g_b: torch.Tensor) -> float:
    """L2 spread: sqrt(||g_a - g_b||^2 / 2), the standard error of one
    estimate summed over voxels."""
    d = (g_a - g_b).double()
    return math.sqrt(0.5 * float(torch.dot(d, d)))


def signal_norm(g_a: torch.Tensor, g_b: torch.Tensor) -> float:
    """Norm of the expected gradient, the noise part of the mean removed
    (0 when the noise dominates)."""
    d = (g_a - g_b).double()
    m = 0.5 * (g_a + g_b).double()
    return math.sqrt(max(float(torch.dot(m, m)) - 0.25 * float(torch.dot(d, d)), 0.0))


def _fresh_grad(paths: N.Paths, beta: torch.Tensor, gt: torch.Tensor, n: int, seed: int, epoch: int,
                images: torch.Tensor, dldi: torch.Tensor, grad: torch.Tensor) -> torch.Tensor:
    paths.store(beta, n, seed, epoch=epoch)
    paths.reweight(beta, images, cache=True)
    N.loss_residual(images, gt, dldi)
    return paths.grad(beta, dldi, grad, cache=True)


def reuse_errors(rec, seed_b: int) -> Dict:
    """Run one recycling window of ``rec`` (a driver.Reconstruction at a
    resample boundary) and return per-step reuse errors and the extinctions
    the window visited.  ``seed_b`` seeds the independent second set."""
    if rec.t % rec.n_r != 0:
        raise ValueError("reuse_errors starts at a resample boundary")
    scene = rec.scene
    pb = N.Paths(scene)
    img = scene.new_images()
    dldi = torch.zeros_like(img)
    gb = torch.zeros_like(rec.grad)
    errs, errs2, sig, betas = [], [], [], []
    for k in range(rec.n_r):
        if k == 0:
            # set B is drawn at the same beta_ref that set A is about to be stored at
            pb.store(rec.beta, rec.n_paths, seed_b, epoch=rec.epoch)
        beta_t = rec.beta.clone()
        pb.reweight(beta_t, img, cache=True)
        N.loss_residual(img, rec.gt, dldi)
        pb.grad(beta_t, dldi, gb, cache=True)
        rec.step()          # set A: the optimisation's own gradient at beta_t
        errs.append(grad_error(rec.grad, gb))
        errs2.append(grad_error_l2(rec.grad, gb))
        sig.append(signal_norm(rec.grad, gb))
        betas.append(beta_t)
    pb.close()
    rms = lambda v: math.sqrt(sum(e * e for e in v) / len(v))
    return {"per_step": errs, "per_step_l2": errs2, "signal": sig, "rms": rms(errs), "rms_l2": rms(errs2),
            "betas": betas}


def resample_errors(scene: N.Scene, gt: torch.Tensor, betas: Sequence[torch.Tensor], budgets: Sequence[int],
                    seeds=(90001, 90002), l2: bool = False) -> Dict[int, float]:
    """RMS over ``betas`` of the fresh-path gradient error at each budget
    (L1 spread, or L2 with ``l2``); both norms in one pass via
    ``resample_errors_both``."""
    return resample_errors_both(scene, gt, betas, budgets, seeds)[1 if l2 else 0]


def resample_errors_both(scene: N.Scene, gt: torch.Tensor, betas: Sequence[torch.Tensor], budgets: Sequence[int],
                         seeds=(90001, 90002)):
    """(L1, L2) fresh-path errors at each budget, RMS over ``betas``."""
    p = N.Paths(scene)
    img = scene.new_images()
    dldi = torch.zeros_like(img)
    ga = torch.zeros(scene.n_voxels, dtype=torch.float64, device=img.device)
    gb = torch.zeros_like(ga)
    out1, out2 = {}, {}
    for n in budgets:
        a1 = a2 = 0.0
        for j, b in enumerate(betas):
            _fresh_grad(p, b, gt, n, seeds[0], j, img, dldi, ga)
            _fresh_grad(p, b, gt, n, seeds[1], j, img, dldi, gb)
            a1 += grad_error(ga, gb) ** 2
            a2 += grad_error_l2(ga, gb) ** 2
        out1[int(n)] = math.sqrt(a1 / len(betas))
        out2[int(n)] = math.sqrt(a2 / len(betas))
    p.close()
    return out1, out2


def rel_errors(g: torch.Tensor, g_ref: torch.Tensor) -> Dict[str, float]:
    """||g - g_ref|| / ||g_ref|| in L2 and in L1, with ||g|| / ||g_ref|| and
    the cosine of the angle between g and g_ref (an estimate that has
    collapsed toward 0 has error near 1 and a small norm ratio)."""
    d = (g - g_ref).double()
    r = g_ref.double()
    gd = g.double()
    rr = max(float(torch.dot(r, r)), 1e-300)
    gg = float(torch.dot(gd, gd))
    return {"l2": math.sqrt(float(torch.dot(d, d)) / rr),
            "l1": float(d.abs().sum()) / max(float(r.abs().sum()), 1e-300),
            "norm_ratio": math.sqrt(gg / rr),
            "cos": float(torch.dot(gd, r)) / math.sqrt(max(gg * rr, 1e-300))}


def tail_share(g: torch.Tensor, g_ref: torch.Tensor, frac: float = 1e-3) -> float:
    """Share of ||g - g_ref||^2 carried by the largest ``frac`` of the voxels'
    squared errors (near frac for a light-tailed error, near 1 when a few
    voxels carry it)."""
    d2 = ((g - g_ref).double()) ** 2
    k = max(1, int(frac * d2.numel()))
    tot = float(d2.sum())
    return float(torch.topk(d2, k).values.sum()) / tot if tot > 0 else 0.0


def reference_gradient(scene: N.Scene, gt: torch.Tensor, beta: torch.Tensor, n: int, copies: int = 16,
                       factor: int = 4, seed: int = 70001, epoch: int = 0, chunk: int = 0) -> torch.Tensor:
    """g_ref(beta): the mean of ``copies`` independent resampled gradients,
    each of ``factor`` x n fresh paths (residual and derivative from the
    same paths, as in the timed step), stored in chunks of ``chunk`` paths
    (default n) normalised by the total."""
    from .driver import ChunkedPaths
    cp = ChunkedPaths(scene, chunk=chunk or n)
    img = scene.new_images()
    dldi = torch.zeros_like(img)
    g = torch.zeros(scene.n_voxels, dtype=torch.float64, device=img.device)
    acc = torch.zeros_like(g)
    for k in range(copies):
        cp.store(beta, factor * n, seed + k, epoch=epoch)
        cp.reweight(beta, img, cache=True)
        N.loss_residual(img, gt, dldi)
        cp.grad(beta, dldi, g, cache=True)
        acc += g
    cp.close()
    return acc / copies


def matched_errors(rec, n_fresh: Sequence[int], ages: Sequence[int], copies: int = 16, factor: int = 4,
                   fresh_draws: int = 2, seed: int = 70001) -> Dict:
    """The reuse and resample gradient errors against a reference gradient.

    ``rec`` (a driver.Reconstruction at a resample boundary, cached
    gradient) runs one recycling window; at each age k in ``ages`` its own
    gradient at beta_t (paths stored k steps earlier) is kept.  Then, per
    kept extinction, g_ref = the mean of ``copies`` fresh gradients of
    ``factor`` x N paths, the reuse error e = ||g - g_ref|| / ||g_ref||, and
    the same error of ``fresh_draws`` fresh-path gradients at each budget of
    ``n_fresh``.  Errors are RMS over the kept ages (and draws), in L2 and in
    L1; with the share of the squared error carried by the largest 0.1% of
    voxels (how heavy the error's tail is)."""
    if rec.t % rec.n_r != 0:
        raise ValueError("matched_errors starts at a resample boundary")
    scene = rec.scene
    kept = []
    for k in range(rec.n_r):
        beta_t = rec.beta.clone()
        rec.step()
        if k in ages:
            kept.append((k, beta_t, rec.grad.clone()))
    p = N.Paths(scene)
    img = scene.new_images()
    dldi = torch.zeros_like(img)
    gf = torch.zeros(scene.n_voxels, dtype=torch.float64, device=img.device)
    keys = ("l2", "l1", "norm_ratio", "cos")
    reuse = {k: [] for k in keys + ("tail",)}
    fresh = {int(m): {k: [] for k in keys + ("tail",)} for m in n_fresh}
    refnorm = []
    for j, (k, b, g) in enumerate(kept):
        g_ref = reference_gradient(scene, rec.gt, b, rec.n_paths, copies, factor, seed + 1000 * j, epoch=j)
        refnorm.append(float(g_ref.double().norm()))
        e = rel_errors(g, g_ref)
        for key in keys:
            reuse[key].append(e[key])
        reuse["tail"].append(tail_share(g, g_ref))
        for m in n_fresh:
            for r in range(fresh_draws):
                _fresh_grad(p, b, rec.gt, int(m), seed + 500 + 17 * r, 100 + j, img, dldi, gf)
                e = rel_errors(gf, g_ref)
                f = fresh[int(m)]
                for key in keys:
                    f[key].append(e[key])
                f["tail"].append(tail_share(gf, g_ref))
    p.close()
    rms = lambda v: math.sqrt(sum(x * x for x in v) / len(v))
    mean = lambda v: sum(v) / len(v)
    out = {"ages": [k for k, _, _ in kept], "copies": copies, "factor": factor, "fresh_draws": fresh_draws,
           "ref_norm_l2": refnorm,
           "reuse": {"l2": rms(reuse["l2"]), "l1": rms(reuse["l1"]), "tail_share_top0.1pct": mean(reuse["tail"]),
                     "norm_ratio": mean(reuse["norm_ratio"]), "cos": mean(reuse["cos"]),
                     "l2_per_age": reuse["l2"], "l1_per_age": reuse["l1"], "norm_ratio_per_age": reuse["norm_ratio"],
                     "cos_per_age": reuse["cos"]},
           "resample": {str(m): {"l2": rms(f["l2"]), "l1": rms(f["l1"]), "tail_share_top0.1pct": mean(f["tail"]),
                                 "norm_ratio": mean(f["norm_ratio"]), "cos": mean(f["cos"])}
                        for m, f in fresh.items()}}
    for norm in ("l2", "l1"):
        fit = n_star(out["reuse"][norm], {m: out["resample"][str(m)][norm] for m in fresh})
        out[f"n_star_{norm}"] = fit["n_star"]
        out[f"slope_{norm}"] = fit["slope"]
    return out


def n_star(e_target: float, errors: Dict[int, float]) -> Dict:
    """Budget of equal error: least-squares line of log e against log n,
    solved for e_target (extrapolated along the fitted line when e_target
    lies outside the swept range)."""
    xs = [math.log(n) for n in errors]
    ys = [math.log(e) for e in errors.values()]
    k = len(xs)
    mx, my = sum(xs) / k, sum(ys) / k
    sxx = sum((x - mx) ** 2 for x in xs)
    slope = sum((x - mx) * (y - my) for x, y in zip(xs, ys)) / sxx
    icpt = my - slope * mx
    return {"n_star": math.exp((math.log(e_target) - icpt) / slope), "slope": slope}
