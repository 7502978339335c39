"""Reuse-vs-resample error matching (Sec. 5): the error measure, the budget
solve, and on the GPU the 1/sqrt(n) law of fresh-path gradients and the
equality of reuse and fresh errors at a resample step."""
import math

import numpy as np
import pytest
import torch

from paper_2110_00085_gb300 import calibrate as CAL


def test_grad_error_closed_form():
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.standard_normal(1000))
    d = torch.from_numpy(0.01 * rng.standard_normal(1000))
    assert CAL.grad_error(x, x) == 0.0 and CAL.grad_error_l2(x, x) == 0.0
    assert abs(CAL.grad_error(x + d, x - d) - 2.0 * float(d.abs().mean())) < 1e-15
    want = math.sqrt(2.0) * float(d.norm())   # sqrt(0.5 |2d|^2)
    assert abs(CAL.grad_error_l2(x + d, x - d) - want) < 1e-12 * want
    # signal norm: |x|^2 + |d|^2 - |d|^2 (mean is x; the noise term removed)
    assert abs(CAL.signal_norm(x + d, x - d) - math.sqrt(float(x.norm()) ** 2 - float(d.norm()) ** 2)) < 1e-9


def test_n_star_recovers_inverse_square_root_law():
    errs = {n: 3.0 / math.sqrt(n) for n in (1 << 10, 1 << 11, 1 << 12, 1 << 13)}
    fit = CAL.n_star(3.0 / math.sqrt(5000.0), errs)
    assert abs(fit["slope"] + 0.5) < 1e-12
    assert abs(fit["n_star"] - 5000.0) < 1e-6 * 5000.0
    # outside the swept range: along the fitted line
    assert abs(CAL.n_star(3.0 / math.sqrt(1 << 15), errs)["n_star"] - (1 << 15)) < 1e-3


@pytest.mark.gpu
def test_fresh_error_halves_when_budget_quadruples_and_reuse_starts_at_it():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    from paper_2110_00085_gb300 import native as N, synth
    from paper_2110_00085_gb300.driver import Reconstruction
    # many contributions per pixel (16^3 grid, 3 cameras of 16^2): the
    # regime where the n^(-1/2) law holds for the L1 spread
    sc = synth.small_scene(n=16, n_cams=3, px=16, peak=20.0, seed=7, n_paths=1 << 18)
    scene = N.Scene(sc)
    beta_gt = torch.from_numpy(sc.beta_cloud.reshape(-1).astype(np.float32)).cuda()
    gt = scene.render_forward(beta_gt, 1 << 20, sc.seed + 5)
    beta0 = torch.full_like(beta_gt, float(sc.beta_cloud.mean()))
    n = sc.n_paths
    rec = Reconstruction(scene, gt, beta0, n, n_r=4, lr=float(sc.beta_cloud.max()) / 50, seed=sc.seed)
    er = CAL.reuse_errors(rec, seed_b=sc.seed + 1)
    assert all(math.isfinite(e) and e > 0 for e in er["per_step"])
    es = CAL.resample_errors(scene, gt, er["betas"], [n // 4, n], seeds=(501, 502))
    ratio = es[n // 4] / es[n]
    # 2 for an n^(-1/2) law (4 for n^(-1), 1 for no decrease); RMS of 4 pairs
    assert 1.3 < ratio < 3.0, ratio
    # at the resample step the reuse gradient is a fresh gradient of n paths
    one = CAL.resample_errors(scene, gt, er["betas"][:1], [n], seeds=(503, 504))[n]
    assert 0.6 < er["per_step"][0] / one < 1.6
