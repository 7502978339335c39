"""The reconstruction schedule of Sec. 6: space carving (the photo-hull
initialisation) matches the oracle's carving voxel by voxel, and the
coarse-to-fine driver lowers the reconstruction error while stepping up
resolution and path budget."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2110_00085_gb300 import native as N
from paper_2110_00085_gb300 import synth
from paper_2110_00085_gb300.driver import CoarseToFine, recon_errors

from _parity import t64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _near_edge(sc, v, tol=1e-3):
    """True when some camera sees the centre of voxel v within tol pixels of
    a pixel edge (float32 and FP64 projections may then disagree)."""
    nx, ny = sc.n[0], sc.n[1]
    ix, iy, iz = v % nx, (v // nx) % ny, v // (nx * ny)
    x = (np.array([ix, iy, iz]) + 0.5) * sc.voxel + np.asarray(sc.origin)
    for c in range(len(sc.cameras)):
        q = O.pixel_coords(sc, c, x)
        if q is not None and np.min(np.abs(q - np.round(q))) < tol:
            return True
    return False


def _assert_masks_match(sc, gpu, orc):
    diff = np.nonzero(gpu != orc)[0]
    assert len(diff) <= max(3, 1e-4 * len(orc)), f"{len(diff)} voxels differ"
    for v in diff:
        assert _near_edge(sc, int(v)), f"voxel {v} differs away from any pixel edge"


def test_space_carving_matches_oracle_on_quadrature_images():
    sc = synth.config(1, n_paths=16)
    img = O.single_scatter_quad(sc.replace(max_orders=1), sc.beta_cloud, sub=4, steps=2)
    thr = 0.05 * img[img > 0].mean()
    orc = O.space_carve(sc, img, thr)
    gpu = N.Scene(sc).space_carve(t64(img), thr).cpu().numpy()
    assert 0 < orc.sum() < orc.size
    _assert_masks_match(sc, gpu, orc)


def test_space_carving_matches_oracle_at_noise128_size():
    """128^3 grid, 15 cameras of 128x128 (the timed workload's geometry),
    on a seeded pattern of cloudy and clear pixels."""
    sc = synth.config(3, n_paths=16)
    npx = sum(c.width * c.height for c in sc.cameras)
    img = (np.random.default_rng(9).uniform(size=npx) < 0.97).astype(np.float64)
    orc = O.space_carve(sc, img, 0.5)
    gpu = N.Scene(sc).space_carve(t64(img), 0.5).cpu().numpy()
    assert 0 < orc.sum() < orc.size
    _assert_masks_match(sc, gpu, orc)


def test_decorrelated_gradient_is_unbiased_where_the_same_set_one_is_not():
    """At 0.7 x the true field (32^3 blobs, 9 cameras of 32x32), along the
    direction of the true field: the mean over 8 path sets of 2^16 of the
    decorrelated gradient (residual of one half, derivative of the other)
    matches the slope of the loss by central differences of fresh renders
    (2^21 paths, independent seeds); the paper's same-set estimator, whose
    expectation adds the gradient of the image variance, does not even
    have the right sign at this budget."""
    from paper_2110_00085_gb300.driver import Reconstruction
    sc = synth.config(1, n_paths=1 << 16)
    scene = N.Scene(sc)
    bt = torch.from_numpy(sc.beta_cloud.reshape(-1).astype(np.float32)).cuda()
    gt = scene.new_images()
    for j in range(8):
        scene.render_forward(bt, 1 << 18, 999, first=j << 18, n_norm=8 << 18, images=gt, accumulate=j > 0)

    def loss(s, seed):
        im = scene.new_images()
        for j in range(2):
            scene.render_forward(bt * s, 1 << 20, seed, first=j << 20, n_norm=1 << 21, images=im, accumulate=j > 0)
        return 0.5 * float(((im - gt) ** 2).sum())

    h = 0.05
    fd = (np.mean([loss(0.7 + h, 100 + r) for r in range(3)]) - np.mean([loss(0.7 - h, 200 + r) for r in range(3)])) / (2 * h)
    dec, same = [], []
    for r in range(8):
        for flag, out in ((True, dec), (False, same)):
            rec = Reconstruction(scene, gt, bt * 0.7, 1 << 16, n_r=1, lr=0.0, seed=300 + r, decorrelate=flag)
            rec.step()
            g = rec.grad * (0.5 if flag else 1.0)      # the decorrelated sum is twice the gradient
            out.append(float(torch.dot(g, bt.double())))
            rec.close()
    torch.cuda.synchronize()
    m, se = np.mean(dec), np.std(dec) / np.sqrt(len(dec))
    assert fd < 0
    assert abs(m - fd) <= 0.3 * abs(fd) + 3 * se, (m, se, fd)
    assert np.mean(same) > 0


def test_coarse_to_fine_reconstruction_moves_toward_the_truth():
    """32^3 blobs, 9 cameras: carved hull at 16x16 pixels, then Alg. 2 at
    16x16 (2^16 paths) and 32x32 (2^18 paths) with the decorrelated
    gradient, optimising the hull only.  The carved start has too much mass
    (the hull is wider than the cloud); the run lowers both the error and
    the mass bias, and voxels outside the hull stay empty."""
    sc = synth.config(1, n_paths=1 << 18)
    beta_true = torch.from_numpy(sc.beta_cloud.reshape(-1).astype(np.float32)).cuda()
    c2f = CoarseToFine(sc, beta_true, levels=[(16, 1 << 16), (32, 1 << 18)], n_r=5,
                       lr=float(beta_true.max()) / 100, window=3, min_gain=0.01, max_steps_per_level=15)
    hist = c2f.run(30)
    hull = c2f.hull.cpu().numpy().astype(bool)
    assert hull[sc.beta_cloud.reshape(-1) > 0.05 * sc.beta_cloud.max()].mean() > 0.99   # the hull holds the cloud
    assert hull.mean() < 0.9                                                       # and is carved
    eps0, delta0 = recon_errors(beta_true, c2f.hull.to(torch.float32) * CoarseToFine.cloud_mean(beta_true))
    assert max(h["level"] for h in hist) == 1
    assert all(np.isfinite([h["loss"], h["eps"], h["delta"]]).all() for h in hist)
    assert np.all(c2f.rec.beta.cpu().numpy()[~hull] == 0.0)
    assert hist[-1]["eps"] < eps0 and abs(hist[-1]["delta"]) < abs(delta0)


def test_reconstruction_reaches_a_stated_error():
    """The same 32^3 field seen by its 9 cameras at 64x64 pixels, 2^24 paths
    per step (512 per voxel), hull carved at 20% of the mean lit pixel, a
    decaying step (max/100 / (1 + k/30)), 150 Adam steps of Alg. 2: the
    relative L1 error falls from about 1.05 to below 0.8 and the mass bias
    stays within 20% (measured: eps 0.72, delta -0.13)."""
    sc = synth.config(1, n_paths=1 << 24)
    beta_true = torch.from_numpy(sc.beta_cloud.reshape(-1).astype(np.float32)).cuda()
    c2f = CoarseToFine(sc, beta_true, levels=[(64, 1 << 24)], n_r=10, lr=float(beta_true.max()) / 100,
                       carve_frac=0.2, min_gain=-1e9, max_steps_per_level=150, lr_decay=30.0)
    hist = c2f.run(150)
    assert len(hist) == 150
    assert hist[0]["eps"] > 0.95
    assert hist[-1]["eps"] < 0.8 and abs(hist[-1]["delta"]) < 0.2


def test_reconstruction_checkpoint_resume_repeats_steps():
    """A snapshot taken at a resample boundary and restored repeats the same
    Adam steps (same paths: seeds and epoch come back with it)."""
    from paper_2110_00085_gb300.driver import Reconstruction
    sc = synth.config(1, n_paths=1 << 14)
    scene = N.Scene(sc)
    bt = torch.from_numpy(sc.beta_cloud.reshape(-1).astype(np.float32)).cuda()
    gt = scene.render_forward(bt, 1 << 15, 999)
    rec = Reconstruction(scene, gt, bt * 0.8, 1 << 14, n_r=3, lr=0.1, seed=5, decorrelate=True)
    for _ in range(3):
        rec.step()
    snap = rec.snapshot()
    for _ in range(4):
        rec.step()
    torch.cuda.synchronize()
    a, la = rec.beta.clone(), float(rec.loss)
    rec.restore(snap)
    for _ in range(4):
        rec.step()
    torch.cuda.synchronize()
    assert torch.allclose(rec.beta, a, rtol=1e-5, atol=1e-6) and abs(float(rec.loss) - la) <= 1e-9 * abs(la)
    assert not torch.equal(snap["beta"], a)
    rec.close()


def test_reconstruction_resumes_from_a_file_checkpoint(tmp_path):
    """save() at a resample boundary and load() into a new Reconstruction of
    the same settings (no stored paths yet) repeat the same Adam steps; a
    checkpoint of other settings is refused."""
    from paper_2110_00085_gb300.driver import Reconstruction
    sc = synth.config(1, n_paths=1 << 14)
    scene = N.Scene(sc)
    bt = torch.from_numpy(sc.beta_cloud.reshape(-1).astype(np.float32)).cuda()
    gt = scene.render_forward(bt, 1 << 15, 999)
    rec = Reconstruction(scene, gt, bt * 0.8, 1 << 14, n_r=3, lr=0.1, seed=5, decorrelate=True)
    # a carved hull: half of the voxels are not optimised
    rec.mask = (torch.arange(scene.n_voxels, device="cuda") % 2).to(torch.uint8)
    for _ in range(3):
        rec.step()
    f = str(tmp_path / "ckpt.pt")
    rec.save(f)
    for _ in range(4):
        rec.step()
    torch.cuda.synchronize()
    a = rec.beta.clone()
    rec.close()
    other = Reconstruction(scene, gt, bt * 0.5, 1 << 14, n_r=3, lr=0.1, seed=5, decorrelate=True)
    other.load(f)
    assert other.mask is not None and torch.equal(other.mask, rec.mask)
    for _ in range(4):
        other.step()
    torch.cuda.synchronize()
    assert torch.allclose(other.beta, a, rtol=1e-5, atol=1e-6)
    # masked voxels kept the loaded extinction
    keep = rec.mask == 0
    assert torch.equal(other.beta[keep], (bt * 0.8)[keep])
    other.close()
    with pytest.raises(ValueError, match="seed"):
        Reconstruction(scene, gt, bt, 1 << 14, n_r=3, lr=0.1, seed=6, decorrelate=True).load(f)
    with pytest.raises(ValueError, match="lr"):
        Reconstruction(scene, gt, bt, 1 << 14, n_r=3, lr=0.2, seed=5, decorrelate=True).load(f)
