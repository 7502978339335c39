"""Reflectometry (Sec. 6): the surface light tracer with a Phong sphere,
stored paths re-evaluated under BRDF parameters, and the gradient in
(kappa, gamma), against the oracle on identical Philox streams."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2110_00085_gb300 import native as N
from paper_2110_00085_gb300 import synth

from _parity import MAX_DIVERGENT, assert_images_close, divergent, t64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _case(n=1 << 16):
    ss = synth.sphere_box(n_paths=n)
    scene = N.SurfScene(ss)
    fp = torch.zeros(n, dtype=torch.int64, device="cuda")
    tal = torch.zeros(N.TALLY_COUNT, dtype=torch.float64, device="cuda")
    paths = N.SurfPaths(scene).store(n, ss.seed, tallies=tal, fingerprints=fp)
    return ss, scene, paths, fp, tal


@pytest.mark.parametrize("kappa,gamma", [(0.7, 50.0), (0.3, 12.0)])
def test_surfaces_images_and_gradient_match_oracle(kappa, gamma):
    ss, scene, paths, fp, tal = _case()
    n = ss.n_paths
    gt = O.surf_render(ss, kappa=0.7, gamma=50.0, seed=ss.seed + 1)["images"]
    img = paths.reweight(kappa, gamma)
    F = img.cpu().numpy()
    dl = F - gt
    g = paths.grad(kappa, gamma, t64(dl))
    ref = O.surf_render(ss, kappa, gamma, dldi=dl, grad_abs=True, fingerprints=True, tallies=True,
                        image_cond=True, grad_cond=True)
    div = divergent(fp, ref["fingerprints"])
    assert len(div) <= max(3, MAX_DIVERGENT * n), f"{len(div)} divergent paths"
    gi, gg = img.clone(), g.clone()
    oi, og = ref["images"].copy(), ref["grad"].copy()
    for p in div:
        one = N.SurfPaths(scene).store(1, ss.seed, first=int(p), n_norm=n)
        gi -= one.reweight(kappa, gamma)
        gg -= one.grad(kappa, gamma, t64(dl))
        r1 = O.surf_render(ss, kappa, gamma, first=int(p), n=1, n_norm=n, dldi=dl)
        oi -= r1["images"]
        og -= r1["grad"]
        one.close()
    torch.cuda.synchronize()
    assert np.abs(oi).max() > 0
    # per pixel 1e-4 plus the float32 budget measured by the oracle (hits near
    # a sphere's silhouette and lobe cosines near the Phong peak are
    # ill-conditioned in any float32 evaluation)
    assert_images_close(gi.cpu().numpy(), oi, cond=ref["image_cond"], what="surface images")
    gg = gg.cpu().numpy()
    assert np.all(np.abs(gg - og) <= 1e-4 * ref["grad_abs"] + ref["grad_cond"]), (gg, og, ref["grad_abs"])
    T = dict(zip(N.TALLY_NAMES, tal.cpu().numpy()))
    for k in ("collisions", "in_view"):
        assert abs(T[k] - ref["tallies"][k]) <= 12 * len(div) + 1


def test_surfaces_reevaluation_is_exact():
    """Stored paths re-evaluated under other parameters and back give the
    same images (only the order of the FP64 additions differs)."""
    ss, scene, paths, fp, tal = _case(1 << 14)
    a = paths.reweight(0.7, 50.0).clone()
    paths.reweight(0.2, 5.0)
    b = paths.reweight(0.7, 50.0)
    torch.cuda.synchronize()
    assert paths.events() > 0
    assert torch.allclose(a, b, rtol=1e-12, atol=0)
