"""The differentiable renderer (torch.autograd.Function over the recycled
forward and render_grad): its backward equals the oracle's gradient of the
same loss on identical path streams, and finite differences of the GPU loss
agree with it (FP32 smoke check)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2110_00085_gb300 import autograd as AG
from paper_2110_00085_gb300 import native as N
from paper_2110_00085_gb300 import synth

from _parity import assert_grad_close, divergent, t32, t64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _setup(n=1 << 12, cfg=1):
    sc = synth.config(cfg, n_paths=n)
    rng = np.random.default_rng(31)
    bt = (sc.beta_cloud * rng.uniform(0.85, 1.2, size=sc.beta_cloud.shape)).astype(np.float32)
    gt = 0.8 * O.render(sc, sc.beta_cloud, n=n, seed=sc.seed + 5)["images"]
    return sc, bt, gt


def test_autograd_backward_matches_oracle():
    sc, bt, gt = _setup()
    n = sc.n_paths
    scene = N.Scene(sc)
    fp = torch.zeros(n, dtype=torch.int64, device="cuda")
    paths = N.Paths(scene).store(t32(sc.beta_cloud), n, sc.seed, fingerprints=fp)
    beta = t32(bt).requires_grad_(True)
    img = AG.render(beta, paths)
    loss = 0.5 * ((img - t64(gt)) ** 2).sum()
    loss.backward()
    F = img.detach().cpu().numpy()
    ref = O.render(sc, sc.beta_cloud, bt, n=n, dldi=F - gt, grad_abs=True, grad_cond=True, fingerprints=True)
    assert len(divergent(fp, ref["fingerprints"])) == 0
    g = beta.grad.double().cpu().numpy()
    assert np.abs(ref["grad"]).max() > 0
    # beta.grad is the float32 rounding of the FP64 sum: 2 u |g| on top
    assert_grad_close(g, ref["grad"], ref["grad_abs"], ref["grad_cond"] + 2.0 * 2 ** -24 * np.abs(ref["grad"]))


def test_autograd_finite_difference_smoke():
    """64^3 blobs in air (two particle types)."""
    sc, bt, gt = _setup(1 << 14, cfg=2)
    n = sc.n_paths
    scene = N.Scene(sc)
    paths = N.Paths(scene).store(t32(sc.beta_cloud), n, sc.seed)
    gtt = t64(gt)
    beta = t32(bt).requires_grad_(True)
    loss = 0.5 * ((AG.render(beta, paths) - gtt) ** 2).sum()
    loss.backward()
    g = beta.grad.double().cpu().numpy()
    order = np.argsort(-np.abs(g))[:6]
    for v in order:
        h = 2e-2 * float(bt.reshape(-1)[v])
        lp = []
        for sgn in (+1, -1):
            b = t32(bt).clone()
            b[v] += sgn * h
            with torch.no_grad():
                lp.append(0.5 * ((paths.reweight(b) - gtt) ** 2).sum().item())
        fd = (lp[0] - lp[1]) / (2 * h)
        assert abs(fd - g[v]) <= 2e-2 * abs(g[v]), (v, fd, g[v])
