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


def test_two_forwards_then_backward_of_the_first():
    """A second forward on the same stored paths replaces the contribution
    cache; the backward of the first must still differentiate the first
    extinction (its cache token is stale, so it re-traces the shadow rays)
    and equal a fresh single forward and backward.  The raw call refuses a
    cached gradient for a grid other than the cached reweight's."""
    sc, bt, gt = _setup()
    n = sc.n_paths
    scene = N.Scene(sc)
    paths = N.Paths(scene).store(t32(sc.beta_cloud), n, sc.seed)
    b1 = t32(bt).requires_grad_(True)
    b2 = t32(bt * 1.1).requires_grad_(True)
    img1 = AG.render(b1, paths)
    tok1 = paths.cache_token()
    img2 = AG.render(b2, paths)
    assert tok1 != 0 and paths.cache_token() not in (0, tok1)
    (0.5 * ((img1 - t64(gt)) ** 2).sum()).backward()
    assert b2.grad is None
    ref_paths = N.Paths(scene).store(t32(sc.beta_cloud), n, sc.seed)
    br = t32(bt).requires_grad_(True)
    img_r = AG.render(br, ref_paths)
    (0.5 * ((img_r - t64(gt)) ** 2).sum()).backward()
    torch.cuda.synchronize()
    assert torch.allclose(img1, img_r, rtol=1e-12, atol=0)
    assert not torch.allclose(img2, img_r, rtol=1e-3, atol=0)
    # re-traced vs cached: the same terms summed in another order (FP32
    # pre-sums of same-voxel terms before the FP64 reductions)
    assert torch.allclose(b1.grad, br.grad, rtol=1e-5, atol=1e-7 * float(br.grad.abs().max()))
    with pytest.raises(RuntimeError, match="another extinction grid"):
        paths.grad(t32(bt * 1.1), t64(gt), cache=True)
    paths.close()
    ref_paths.close()


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


def test_autograd_backward_equals_oracle_central_differences_64_voxels():
    """64^3 blobs in air: the backward of the differentiable renderer on 64
    voxels drawn with seed 3 among those with beta >= 1 /km equals central
    differences (h = 1e-4 beta_v) of the oracle's FP64 loss on the same
    fixed paths (the recycled estimator is smooth in beta with the paths
    fixed, and its exact derivative is the score-function gradient)."""
    n = 1 << 13
    sc, bt, gt = _setup(n, cfg=2)
    scene = N.Scene(sc)
    fp = torch.zeros(n, dtype=torch.int64, device="cuda")
    paths = N.Paths(scene).store(t32(sc.beta_cloud), n, sc.seed, fingerprints=fp)
    beta = t32(bt).requires_grad_(True)
    img = AG.render(beta, paths)
    loss = 0.5 * ((img - t64(gt)) ** 2).sum()
    loss.backward()
    g = beta.grad.double().cpu().numpy()
    F = img.detach().cpu().numpy()
    ref = O.render(sc, sc.beta_cloud, bt, n=n, dldi=F - gt, grad_abs=True, grad_cond=True, fingerprints=True)
    assert len(divergent(fp, ref["fingerprints"])) == 0
    flat = bt.reshape(-1)
    cand = np.nonzero(flat >= 1.0)[0]
    vox = np.random.default_rng(3).choice(cand, 64, replace=False)

    def oracle_loss(b):
        im = O.render(sc, sc.beta_cloud, b, n=n, threads=8)["images"]
        return 0.5 * float(np.sum((im - gt) ** 2))

    fd = np.zeros(64)
    for i, v in enumerate(vox):
        h = 1e-4 * float(flat[v])
        lp = []
        for sgn in (+1, -1):
            b = flat.astype(np.float64).copy()
            b[v] += sgn * h
            lp.append(oracle_loss(b.astype(np.float32).reshape(bt.shape)))
        # the grid is float32: use the step that float32 actually took
        hp = float(np.float32(flat[v] + h)) - float(flat[v])
        hm = float(flat[v]) - float(np.float32(flat[v] - h))
        fd[i] = (lp[0] - lp[1]) / (hp + hm)
    # per voxel: 1e-4 of the voxel's term mass, the float32 budget, float32
    # rounding of beta.grad, and the FD's FP64 roundoff (|L| 1e-15 / 2h)
    L = oracle_loss(bt)
    tol = (1e-4 * ref["grad_abs"][vox] + ref["grad_cond"][vox] + 2.0 * 2 ** -24 * np.abs(g[vox])
           + 1e-15 * abs(L) / (2e-4 * flat[vox].astype(np.float64)))
    err = np.abs(g[vox] - fd)
    assert np.abs(fd).max() > 0
    assert (err <= tol).all(), [(int(v), g[v], f, t) for v, f, e, t in zip(vox, fd, err, tol) if e > t]


def test_autograd_central_differences_fullsize_64_voxels():
    """The differentiable renderer at the full size of the 64^3 blobs-in-air
    workload (9 cameras of 64x64, 2^22 stored paths): the backward against
    central differences of the same renderer's FP64-summed loss, on 64 voxels
    drawn with seed 5 among those with beta >= 1 /km.  With the paths fixed
    the recycled estimate is smooth in beta, so the differences converge to
    the score-function gradient; what separates them is the O(h^2)
    truncation and the FP32 rounding of the perturbed terms (a few 1e-6 of
    the voxel's share of the loss)."""
    sc = synth.config(2)
    n = sc.n_paths
    assert n == 1 << 22
    scene = N.Scene(sc)
    bt = (sc.beta_cloud * np.random.default_rng(41).uniform(0.85, 1.2, size=sc.beta_cloud.shape)).astype(np.float32)
    gt = scene.render_forward(t32(sc.beta_cloud), n, sc.seed + 5)       # the target: the true cloud, other paths
    paths = N.Paths(scene).store(t32(sc.beta_cloud), n, sc.seed)
    beta = t32(bt).requires_grad_(True)
    loss = 0.5 * ((AG.render(beta, paths) - gt) ** 2).sum()
    loss.backward()
    g = beta.grad.double().cpu().numpy()
    flat = bt.reshape(-1)
    vox = np.random.default_rng(5).choice(np.nonzero(flat >= 1.0)[0], 64, replace=False)
    fd = np.zeros(64)
    with torch.no_grad():
        for i, v in enumerate(vox):
            h = 1e-2 * float(flat[v])
            lp = []
            for sgn in (+1, -1):
                b = t32(bt)
                b[v] += sgn * h
                lp.append(0.5 * float(((paths.reweight(b) - gt) ** 2).sum()))
            hp = float(np.float32(flat[v] + h)) - float(flat[v])
            hm = float(flat[v]) - float(np.float32(flat[v] - h))
            fd[i] = (lp[0] - lp[1]) / (hp + hm)
    gv = g[vox]
    rel = np.abs(fd - gv) / np.maximum(np.abs(gv), 1e-300)
    print(f"64 voxels at 2^22 paths: |g| {np.abs(gv).min():.3e}..{np.abs(gv).max():.3e}; relative FD difference "
          f"median {np.median(rel):.2e}, max {rel.max():.2e}")
    assert np.abs(gv).min() > 0
    tol = 2e-3 * np.abs(gv) + 1e-5 * np.abs(gv).max()
    assert (np.abs(fd - gv) <= tol).all(), [(int(v), a, b) for v, a, b, e, t in
                                            zip(vox, gv, fd, np.abs(fd - gv), tol) if e > t]
    assert np.median(rel) < 2e-4
    paths.close()
