"""Gradient error of path reuse vs resampling, and the resample path budget
of equal error (Sec. 5: recycled paths trade variance for speed).

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
