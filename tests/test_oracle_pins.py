"""Pins of the FP64 CPU oracle against facts the paper and mathematics fix.

Nothing here compares the oracle with itself or with the CUDA path: every
check is a published known answer, a closed form, an invariant, a special
case or brute force.  Each test names the part of the oracle it pins.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2110_00085_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ---
def test_philox_known_answers():
    """Random123 known-answer vectors for Philox4x32-10 (Salmon et al. SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_fnv_offset_basis():
    """FNV-1a 64 of the empty input is the published offset basis."""
    assert O.fnv1a_words([]) == 0xCBF29CE484222325


# --------------------------------------------------------- phase functions --
@pytest.mark.parametrize("g", [0.0, 0.5, 0.85, -0.3])
def test_hg_normalised_and_mean_cosine(g):
    """HG integrates to 1 over the sphere (Eq. phase_conservation) and its
    mean cosine equals its asymmetry parameter g."""
    norm = 2 * math.pi * integrate.quad(lambda m: O.phase_hg(g, m), -1, 1, limit=200, epsabs=1e-13)[0]
    mean = 2 * math.pi * integrate.quad(lambda m: m * O.phase_hg(g, m), -1, 1, limit=200, epsabs=1e-13)[0]
    assert abs(norm - 1) < 1e-9
    assert abs(mean - g) < 1e-9


def test_hg_isotropic_special_case():
    for mu in (-1, -0.3, 0, 0.7, 1):
        assert abs(O.phase_hg(0.0, mu) - 1 / (4 * math.pi)) < 1e-15


def test_rayleigh_moments():
    """Rayleigh: normalised, mean cosine 0, <mu^2> = 2/5."""
    f = O.phase_rayleigh
    n = 2 * math.pi * integrate.quad(f, -1, 1)[0]
    m1 = 2 * math.pi * integrate.quad(lambda m: m * f(m), -1, 1)[0]
    m2 = 2 * math.pi * integrate.quad(lambda m: m * m * f(m), -1, 1)[0]
    assert abs(n - 1) < 1e-12 and abs(m1) < 1e-12 and abs(m2 - 0.4) < 1e-12


@pytest.mark.parametrize("g", [0.85, 0.5, -0.4])
def test_hg_sampler_inverts_cdf(g):
    """The HG sampler is the inverse of the closed-form HG CDF in mu."""
    def cdf(mu):
        return (1 - g * g) / (2 * g) * (1 / math.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))
    for u in np.linspace(1e-6, 1, 101):
        assert abs(cdf(O.sample_hg(g, u)) - u) < 1e-9


def test_rayleigh_sampler_inverts_cdf():
    """Rayleigh CDF in mu is (mu^3 + 3 mu + 4)/8; the sampler inverts it."""
    for u in np.linspace(1e-6, 1, 101):
        mu = O.sample_rayleigh(u)
        assert abs((mu ** 3 + 3 * mu + 4) / 8 - u) < 1e-12


def test_sampler_cdf_matches_pdf_integral():
    """The sampled distribution's CDF equals the integral of the pdf the
    estimator divides by (ties the sampler to the evaluated phase)."""
    g = 0.85
    for u in (0.1, 0.5, 0.9, 0.99):
        mu = O.sample_hg(g, u)
        F = 2 * math.pi * integrate.quad(lambda m: O.phase_hg(g, m), -1, mu, limit=200, epsabs=1e-13)[0]
        assert abs(F - u) < 1e-8
        mu = O.sample_rayleigh(u)
        F = 2 * math.pi * integrate.quad(O.phase_rayleigh, -1, mu)[0]
        assert abs(F - u) < 1e-12


# ------------------------------------------------------ directions, bases --
def test_onb_orthonormal_right_handed():
    rng = np.random.default_rng(0)
    ns = [np.array(v, float) for v in [(0, 0, 1), (0, 0, -1), (1, 0, 0), (0, 1, 0)]]
    ns += [v / np.linalg.norm(v) for v in rng.normal(size=(50, 3))]
    for n in ns:
        b1, b2 = O.onb(n)
        M = np.stack([b1, b2, n])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-12)
        assert np.allclose(np.cross(b1, b2), n, atol=1e-12)


def test_rotation_sets_polar_and_azimuth():
    rng = np.random.default_rng(1)
    for _ in range(50):
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        mu = rng.uniform(-1, 1); phi = rng.uniform(0, 2 * math.pi)
        o = O.rotate(d, mu, phi)
        b1, b2 = O.onb(d)
        st = math.sqrt(1 - mu * mu)
        assert abs(np.linalg.norm(o) - 1) < 1e-12
        assert abs(o @ d - mu) < 1e-12
        assert abs(o @ b1 - st * math.cos(phi)) < 1e-12
        assert abs(o @ b2 - st * math.sin(phi)) < 1e-12


# ------------------------------------------------------------- cameras ------
def test_pixel_solid_angles_tile_the_image():
    """Pixel solid angles add up to the image rectangle's solid angle, and the
    whole plane (tan -> inf) is a hemisphere, 2 pi."""
    tx, ty, W, H = 0.6, 0.45, 24, 18
    tot = sum(O.pixel_solid_angle(tx, ty, W, H, c, r) for c in range(W) for r in range(H))
    full = 4 * math.atan(tx * ty / math.sqrt(1 + tx * tx + ty * ty))
    assert abs(tot - full) < 1e-12
    assert abs(O.pixel_solid_angle(1e9, 1e9, 1, 1, 0, 0) - 2 * math.pi) < 1e-6


def test_small_pixel_solid_angle_is_area_cos3():
    """A tiny pixel at image-plane position (x, y) subtends area*cos^3."""
    tx = ty = 0.5
    W = H = 2001
    for c, r in [(1000, 1000), (1800, 300), (50, 1950)]:
        om = O.pixel_solid_angle(tx, ty, W, H, c, r)
        x = tx * (-1 + 2 * (c + 0.5) / W)
        y = ty * (1 - 2 * (r + 0.5) / H)
        area = (2 * tx / W) * (2 * ty / H)
        cos3 = (1 + x * x + y * y) ** -1.5
        assert abs(om / (area * cos3) - 1) < 1e-5


def test_camera_frame():
    sc = synth.config(1, n_paths=16)
    for i, cam in enumerate(sc.cameras):
        f = O.camera_frame(sc, i)
        fwd = np.subtract(cam.look_at, cam.pos); fwd /= np.linalg.norm(fwd)
        assert np.allclose(f["F"], fwd, atol=1e-6)
        assert abs(f["R"] @ f["F"]) < 1e-12 and abs(f["U"] @ f["F"]) < 1e-12
        assert f["U"] @ np.array(cam.up) > 0
        assert abs(f["ty"] - math.tan(float(np.float32(cam.fov_y)) / 2)) < 1e-12


# --------------------------------------------------- grid traversal (DDA) ---
def _grid_scene(n=8, voxel=0.02):
    return synth.Scene(name="g", n=(n, n, n), voxel=voxel, beta_cloud=np.zeros((n, n, n), np.float32))


def test_intervals_axis_ray():
    sc = _grid_scene()
    d = 0.02
    vox, ln = O.intervals(sc, (-0.1, 2.5 * d, 5.5 * d), (1, 0, 0), 10.0)
    assert len(vox) == 8
    assert np.allclose(ln, d)
    assert list(vox) == [i + 8 * (2 + 8 * 5) for i in range(8)]


def test_intervals_main_diagonal_through_corners():
    """A ray through voxel corners: every interval is a full diagonal and
    zero-length crossings are dropped."""
    sc = _grid_scene()
    d = 0.02
    u = np.ones(3) / math.sqrt(3)
    vox, ln = O.intervals(sc, -0.1 * u, u, 10.0)
    assert len(vox) == 8
    assert np.allclose(ln, math.sqrt(3) * d)
    assert list(vox) == [i * (1 + 8 + 64) for i in range(8)]


def test_optical_depth_matches_dense_sampling():
    """Sum beta*l over intervals equals a dense midpoint integral of the
    piecewise-constant field along random rays (brute force)."""
    rng = np.random.default_rng(3)
    n = 8
    beta = rng.uniform(0, 30, size=(n, n, n)).astype(np.float32)
    sc = synth.Scene(name="g", n=(n, n, n), voxel=0.02, beta_cloud=beta, beta_air=0.5)
    L = n * 0.02
    for _ in range(20):
        p = rng.uniform(-0.05, L + 0.05, size=3)
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        tmax = rng.uniform(0.05, 0.4)
        tau = -math.log(O.transmittance(sc, beta, p, d, tmax))
        m = 400000
        t = (np.arange(m) + 0.5) * (tmax / m)
        x = p[None, :] + t[:, None] * d[None, :]
        inside = np.all((x >= 0) & (x < L), axis=1)
        idx = np.floor(x[inside] / 0.02).astype(int)
        b = beta[idx[:, 2], idx[:, 1], idx[:, 0]].astype(np.float64) + 0.5
        ref = b.sum() * (tmax / m)
        vox, ln = O.intervals(sc, p, d, tmax)
        assert abs(ln.sum() - inside.sum() * tmax / m) < 3e-6
        assert abs(tau - ref) <= 2e-5 * max(ref, 1.0)


# ------------------------------------------------------------- sun source ---
def test_sun_rectangle_hit_fraction():
    """Start points are uniform on the sun rectangle: the fraction that
    enters the box equals the box's projected area over the rectangle's
    area (projected area of a box along s: sum over axes of the face
    area times |s_axis|)."""
    n = 16
    sc = synth.Scene(name="s", n=(n, 8, 4), voxel=0.02,
                     beta_cloud=np.zeros((4, 8, n), np.float32),
                     sun_dir=synth.sun_from_zenith(40.0, 25.0), n_paths=1 << 16,
                     cameras=synth.arc_cameras(1, (n * 0.02, 0.16, 0.08), 4, 4))
    Lx, Ly, Lz = sc.box_size
    s = np.abs(np.array(sc.sun_dir))
    proj = Ly * Lz * s[0] + Lx * Lz * s[1] + Lx * Ly * s[2]
    rect = O.sun_rect(sc)
    p = proj / rect["area"]
    r = O.render(sc, sc.beta_cloud, tallies=True)
    frac = r["tallies"]["entered"] / sc.n_paths
    sig = math.sqrt(p * (1 - p) / sc.n_paths)
    assert abs(frac - p) < 4 * sig
    w0 = rect["area"] * sc.sun_irradiance
    assert abs(r["tallies"]["injected"] + r["tallies"]["missed"] - w0 * sc.n_paths) < 1e-9 * w0 * sc.n_paths


# ------------------------------------------------------------ closed forms --
def test_beer_lambert_pure_absorber():
    """P-a: an absorbing cube (albedo 0) lit from the zenith: the escaping
    weight fraction is exp(-beta L) (binomial 4 sigma); images are 0."""
    n = 8
    beta = np.full((n, n, n), 5.0, np.float32)
    sc = synth.Scene(name="bl", n=(n, n, n), voxel=0.02, beta_cloud=beta, albedo_cloud=0.0,
                     sun_dir=(0.0, 0.0, -1.0), n_paths=1 << 15,
                     cameras=synth.arc_cameras(3, (0.16,) * 3, 8, 8))
    r = O.render(sc, beta, tallies=True)
    T = r["tallies"]
    p = math.exp(-5.0 * 0.16)
    frac = T["escaped"] / T["injected"]
    sig = math.sqrt(p * (1 - p) / T["entered"])
    assert abs(frac - p) < 4 * sig
    assert np.all(r["images"] == 0.0)


def _slab_scene(n_paths):
    nxy, nz = 64, 2
    beta = np.full((nz, nxy, nxy), 10.0, np.float32)
    box = (nxy * 0.02, nxy * 0.02, nz * 0.02)
    return synth.Scene(name="slab", n=(nxy, nxy, nz), voxel=0.02, beta_cloud=beta,
                       albedo_cloud=0.99, hg_g=0.85, sun_dir=synth.sun_from_zenith(30.0),
                       cameras=synth.arc_cameras(1, box, 16, 16), max_orders=1, rr_start=5,
                       n_paths=n_paths)


def test_homogeneous_slab_single_scattering():
    """P-b: first-order radiance of a laterally infinite homogeneous slab,
    L = w F0 p(Theta) mu0/(mu0+mu) [1 - exp(-tau*(1/mu0+1/mu))] (first-order
    term of the integrated RTE of Sec. 3.2 for a collimated source); central
    pixels of a wide thin slab, within 1% + 4 sigma."""
    sc = _slab_scene(1 << 20)
    r = O.render(sc, sc.beta_cloud, threads=8)
    img = r["images"].reshape(16, 16)
    f = O.camera_frame(sc, 0)
    s = np.array(sc.sun_dir)
    mu0 = -s[2]
    tau = 10.0 * 0.04
    vals, exp_ = [], []
    for row in range(6, 10):
        for col in range(6, 10):
            x = f["tx"] * (-1 + 2 * (col + 0.5) / 16)
            y = f["ty"] * (1 - 2 * (row + 0.5) / 16)
            d = f["F"] + x * f["R"] + y * f["U"]
            d /= np.linalg.norm(d)
            mu = -d[2]
            cth = -(s @ d)
            Lx = 0.99 * sc.sun_irradiance * O.phase_hg(0.85, cth) * mu0 / (mu0 + mu) * (
                1 - math.exp(-tau * (1 / mu0 + 1 / mu)))
            vals.append(img[row, col]); exp_.append(Lx)
    vals = np.array(vals); exp_ = np.array(exp_)
    ratio = vals.sum() / exp_.sum()
    assert abs(ratio - 1) < 0.01 + 4 * (np.std(vals / exp_) / math.sqrt(len(vals)))


def _batch_images(sc, beta_ref, beta_t=None, blocks=16, seed=None, threads=8):
    n = sc.n_paths // blocks
    ims = []
    for b in range(blocks):
        r = O.render(sc, beta_ref, beta_t, first=b * n, n=n, threads=threads, seed=seed)
        ims.append(r["images"])
    ims = np.array(ims)
    return ims.mean(0), ims.std(0, ddof=1) / math.sqrt(blocks)


def test_single_scatter_quadrature_matches_first_order_mc():
    """P-c: first-order Monte Carlo (max_orders = 1) equals a deterministic
    quadrature of the first-order radiance on the same grid.  Pixels whose
    quadrature is not converged (box edges) are excluded."""
    sc = synth.small_scene(n=8, n_cams=2, px=12, peak=20.0, seed=11, n_paths=1 << 18)
    sc = sc.replace(max_orders=1)
    q_fine = O.single_scatter_quad(sc, sc.beta_cloud, sub=24, steps=8)
    q_coarse = O.single_scatter_quad(sc, sc.beta_cloud, sub=12, steps=4)
    mc, sd = _batch_images(sc, sc.beta_cloud)
    use = q_fine > 0.05 * q_fine.max()
    assert use.sum() >= 30
    z = (mc[use] - q_fine[use]) / np.sqrt(sd[use] ** 2 + (q_fine[use] - q_coarse[use]) ** 2)
    assert np.mean(z ** 2) < 2.5
    assert np.max(np.abs(z)) < 5.0


# --------------------------------------------------------------- invariants --
def test_energy_balance_exact():
    """P-d: injected + roulette gain = escaped + absorbed + truncated +
    roulette-killed, per path, to FP64 rounding."""
    for sc in (synth.config(1, n_paths=1 << 12), synth.config(2, n_paths=1 << 10)):
        T = O.render(sc, sc.beta_cloud, tallies=True)["tallies"]
        lhs = T["injected"] + T["rr_gain"]
        rhs = T["escaped"] + T["absorbed"] + T["truncated"] + T["rr_killed"]
        assert abs(lhs - rhs) < 1e-11 * lhs


def test_conservative_medium_no_roulette():
    """P-d at albedo 1 without roulette: what enters leaves (or is cut by the
    order limit); nothing is absorbed."""
    sc = synth.small_scene(n=8, n_cams=1, px=4, peak=5.0, seed=5, n_paths=1 << 12)
    sc = sc.replace(albedo_cloud=1.0, max_orders=60, rr_start=100)
    T = O.render(sc, sc.beta_cloud, tallies=True)["tallies"]
    assert T["absorbed"] == 0.0 and T["rr_gain"] == 0.0
    assert abs(T["escaped"] + T["truncated"] - T["injected"]) < 1e-11 * T["injected"]
    assert T["truncated"] < 1e-3 * T["injected"]


def test_recycling_ratio_is_one_at_reference():
    """P-e (exact part): paths reused under the very extinction they were
    drawn from reproduce the plain estimate bit for bit (r == 1)."""
    sc = synth.small_scene(n=8, n_cams=3, px=8, seed=3, n_paths=1 << 10)
    a = O.render(sc, sc.beta_cloud)["images"]
    b = O.render(sc, sc.beta_cloud, sc.beta_cloud.copy())["images"]
    assert np.array_equal(a, b)


def test_recycled_estimator_unbiased():
    """P-e: paths drawn under M_ref, reweighted to M_t, estimate the same
    images as paths drawn under M_t (importance sampling is unbiased,
    Appendix A) -- independent seeds, batch-means z-scores."""
    sc = synth.small_scene(n=8, n_cams=3, px=6, seed=9, n_paths=1 << 16)
    rng = np.random.default_rng(4)
    bt = (sc.beta_cloud * rng.uniform(0.8, 1.3, size=sc.beta_cloud.shape)).astype(np.float32)
    m1, s1 = _batch_images(sc, sc.beta_cloud, bt, seed=101)
    m2, s2 = _batch_images(sc, bt, None, seed=202)
    ok = (m1 + m2) > 1e-3 * (m1 + m2).max()
    z = (m1[ok] - m2[ok]) / np.sqrt(s1[ok] ** 2 + s2[ok] ** 2)
    assert np.mean(z ** 2) < 2.0
    assert np.max(np.abs(z)) < 5.0
    # camera totals (lower variance)
    tot1, tot2 = m1.sum(), m2.sum()
    assert abs(tot1 - tot2) < 4 * math.sqrt((s1 ** 2).sum() + (s2 ** 2).sum()) + 0.0


# --------------------------------------------------- gradient (FD identity) --
def _fd_scene(air):
    n = 4
    rng = np.random.default_rng(21 + air)
    beta = rng.uniform(2.0, 12.0, size=(n, n, n)).astype(np.float32)
    return synth.Scene(name="fd", n=(n, n, n), voxel=0.04, beta_cloud=beta,
                       beta_air=0.6 if air else 0.0, albedo_air=0.9, albedo_cloud=0.95,
                       cameras=synth.arc_cameras(2, (0.16,) * 3, 4, 4),
                       n_paths=1 << 11, seed=77)


@pytest.mark.parametrize("air", [0, 1])
def test_gradient_equals_finite_difference_4cubed(air):
    """P-f: with paths fixed, F(M_t | M_ref) is smooth in M_t and the paper's
    recycled gradient estimator (Eq. 21 with the PSF of Sec. 4.4) is its exact
    derivative; central differences of the FP64 loss on every voxel of a 4^3
    grid (brute force), with air (two particle types) and without."""
    sc = _fd_scene(air)
    rng = np.random.default_rng(5)
    bref = sc.beta_cloud
    bt = (bref * rng.uniform(0.85, 1.2, size=bref.shape)).astype(np.float32)
    igt = 0.7 * O.render(sc, bref, seed=999)["images"]

    def loss(b):
        F = O.render(sc, bref, b)["images"]
        return 0.5 * np.sum((F - igt) ** 2)

    F = O.render(sc, bref, bt)["images"]
    r = O.render(sc, bref, bt, dldi=F - igt, grad_abs=True)
    g, ga = r["grad"], r["grad_abs"]
    flat = bt.reshape(-1)
    assert np.abs(g).max() > 0
    for v in range(flat.size):
        bp = flat.copy(); bm = flat.copy()
        bp[v] = np.float32(flat[v] * (1 + 1e-3)); bm[v] = np.float32(flat[v] * (1 - 1e-3))
        fd = (loss(bp) - loss(bm)) / (float(bp[v]) - float(bm[v]))
        assert abs(fd - g[v]) <= 1e-6 * ga[v] + 1e-14, (v, fd, g[v], ga[v])


def test_threads_do_not_change_results():
    sc = synth.config(1, n_paths=1 << 11)
    a = O.render(sc, sc.beta_cloud, threads=1)["images"]
    b = O.render(sc, sc.beta_cloud, threads=4)["images"]
    assert np.allclose(a, b, rtol=1e-12, atol=1e-15)


def test_fingerprints_identify_paths():
    sc = synth.config(1, n_paths=1 << 10)
    f1 = O.render(sc, sc.beta_cloud, fingerprints=True)["fingerprints"]
    f2 = O.render(sc, sc.beta_cloud, fingerprints=True)["fingerprints"]
    f3 = O.render(sc, sc.beta_cloud, fingerprints=True, seed=sc.seed + 1)["fingerprints"]
    assert np.array_equal(f1, f2)
    # paths that never collide share one fingerprint; the rest are distinct
    assert np.mean(f1 != f3) > 0.25
    assert len(np.unique(f1)) > 0.25 * len(f1)


# ------------------------------------------------ float32 image budget ------
def test_image_budget_is_measured_not_injected():
    """image_cond (the parity tolerance's float32 term) is test
    infrastructure: asking for it leaves the images untouched, it is
    non-negative and does not depend on the thread split, it is small where
    the geometry is smooth (blob cloud, no air), and it is large for a path
    whose last collision lies in thin air just past cloud edges (perturbing
    its vertices by a float32 roundoff moves the collision far)."""
    sc = synth.config(1, n_paths=1 << 10)
    plain = O.render(sc, sc.beta_cloud)
    r1 = O.render(sc, sc.beta_cloud, image_cond=True)
    r4 = O.render(sc, sc.beta_cloud, image_cond=True, threads=4)
    assert np.array_equal(plain["images"], r1["images"])
    ic, im = r1["image_cond"], r1["images"]
    assert (ic >= 0).all()
    assert np.allclose(ic, r4["image_cond"], rtol=1e-12, atol=1e-300)
    lit = im > 0
    assert lit.sum() > 100
    # about 1e-5 of a pixel, mostly the float32 running sums of the optical
    # depths (u times the sum of their partial sums), well below the 1e-4
    # tolerance it is added to
    assert np.median(ic[lit] / im[lit]) < 3e-5
    # thresholded cloud with air: one path with a thin-air last collision
    c = synth.config(2, n_paths=1 << 11).replace(cameras=synth.arc_cameras(7, (1.28,) * 3, 40, 40))
    br = c.beta_cloud.astype(np.float32)
    one = O.render(c, br, first=718, n=1, n_norm=2048, image_cond=True, scene_id=2)
    k = 2 * 40 * 40 + 788      # camera 2: the local estimate of its 4th collision
    assert one["images"][k] > 0
    assert one["image_cond"][k] > 100 * np.median(ic[lit] / im[lit]) * one["images"][k]


# ------------------------------------------------------------ space carving --
def test_space_carving_limits_and_monotonicity():
    """Photo-hull of the initialisation (Sec. 6): all-cloudy images keep
    every voxel, all-clear ones carve every voxel (each camera's field of
    view holds the whole box); a higher threshold and an extra camera can
    only carve more."""
    sc = synth.config(1, n_paths=16)
    npx = sum(c.width * c.height for c in sc.cameras)
    V = int(np.prod(sc.n))
    assert O.space_carve(sc, np.ones(npx), 0.5).sum() == V
    assert O.space_carve(sc, np.zeros(npx), 0.0).sum() == 0
    img = O.single_scatter_quad(sc.replace(max_orders=1), sc.beta_cloud, sub=4, steps=2)
    lo = O.space_carve(sc, img, 0.02 * img.max())
    hi = O.space_carve(sc, img, 0.2 * img.max())
    assert hi.sum() < lo.sum() and not np.any(hi & ~lo)
    few = sc.replace(cameras=sc.cameras[:4])
    m4 = O.space_carve(few, img[: sum(c.width * c.height for c in few.cameras)], 0.02 * img.max())
    assert not np.any(lo & ~m4) and m4.sum() > lo.sum()


def test_space_carving_keeps_the_cloud_of_single_scatter_images():
    """Images of the deterministic single-scattering quadrature (independent
    of the carving code) of a blob cloud without air, carved at threshold 0:
    every voxel with extinction is kept (its own line of sight to each
    camera crosses cloud, lit by the sun), and the hull is much smaller than
    the grid."""
    sc = synth.config(1, n_paths=16)
    beta = sc.beta_cloud.copy()
    beta[beta < 0.05 * beta.max()] = 0.0          # a cloud with an edge
    img = O.single_scatter_quad(sc.replace(max_orders=1), beta, sub=8, steps=2)
    mask = O.space_carve(sc, img, 0.0)
    cloud = beta.reshape(-1) > 0
    assert cloud.any()
    assert np.all(mask[cloud] == 1)
    assert mask.sum() < 0.5 * mask.size


# ------------------------------------------------------------ reflectometry --
def test_surfaces_energy_balance_and_diffuse_limit():
    """Closed box (Sec. 6 reflectometry stand-in): injected = escaped +
    absorbed (Phong factors below 1) + truncated + roulette, to FP64
    rounding; with kappa = 0 the images do not depend on gamma and the
    gamma derivative is exactly 0."""
    ss = synth.sphere_box(n_paths=1 << 14)
    r = O.surf_render(ss, tallies=True)
    T = r["tallies"]
    lhs = T["injected"] + T["rr_gain"]
    rhs = T["escaped"] + T["absorbed"] + T["truncated"] + T["rr_killed"]
    assert abs(lhs - rhs) < 1e-10 * lhs and T["absorbed"] > 0
    a = O.surf_render(ss, kappa=0.0, gamma=5.0)["images"]
    b = O.surf_render(ss, kappa=0.0, gamma=80.0, dldi=np.ones(ss.n_pixels))
    assert np.array_equal(a, b["images"])
    assert b["grad"][1] == 0.0 and b["grad"][0] != 0.0


def test_surfaces_gradient_equals_finite_differences():
    """Paths do not depend on (kappa, gamma), so the gradient of the loss
    is the exact derivative of the fixed-path estimate: central differences
    of the FP64 loss in kappa and in gamma."""
    ss = synth.sphere_box(n_paths=1 << 12)
    gt = O.surf_render(ss, kappa=0.7, gamma=50.0)["images"]
    k0, g0 = 0.4, 20.0
    F = O.surf_render(ss, kappa=k0, gamma=g0)["images"]
    r = O.surf_render(ss, kappa=k0, gamma=g0, dldi=F - gt, grad_abs=True)

    def loss(k, g):
        return 0.5 * float(np.sum((O.surf_render(ss, kappa=k, gamma=g)["images"] - gt) ** 2))

    for j, (h, args) in enumerate(((1e-5, lambda e: (k0 + e, g0)), (1e-3, lambda e: (k0, g0 + e)))):
        fd = (loss(*args(h)) - loss(*args(-h))) / (2 * h)
        assert abs(fd - r["grad"][j]) <= 1e-6 * r["grad_abs"][j], (j, fd, r["grad"][j])


def _view_factor_square(px, py, x0, x1, y0, y1, h=1.0):
    """View factor from a floor point to the parallel rectangle [x0,x1] x
    [y0,y1] at height h (Lambertian): sum of four corner rectangles."""
    def f(a, b):
        sa, sb = math.sqrt(a * a + h * h), math.sqrt(b * b + h * h)
        return (a / sa * math.atan(b / sa) + b / sb * math.atan(a / sb)) / (2.0 * math.pi)
    return f(x1 - px, y1 - py) - f(x0 - px, y1 - py) - f(x1 - px, y0 - py) + f(x0 - px, y0 - py)


def test_surfaces_first_order_floor_radiance_closed_form():
    """No spheres, first order only: the floor's radiance is the emitter's
    radiance times the view factor to the emitter (diffuse, no absorption),
    so pixels that see the floor average to the closed form."""
    ss = synth.sphere_box(n_paths=1 << 21).replace(spheres=np.zeros((0, 4)), phong=-1, max_orders=1)
    img = O.surf_render(ss)["images"].reshape(ss.camera.height, ss.camera.width)
    # closed form per pixel: floor points on a fine grid, binned by pixel
    acc = np.zeros_like(img); cnt = np.zeros_like(img)
    for xx in np.linspace(0.005, 0.995, 120):
        for yy in np.linspace(0.005, 0.995, 120):
            q = O.pixel_coords(_surf_as_scene(ss), 0, (xx, yy, 0.0))
            if q is None:
                continue
            c, rr = int(q[0]), int(q[1])
            if 0 <= c < ss.camera.width and 0 <= rr < ss.camera.height:
                acc[rr, c] += ss.radiance * _view_factor_square(xx, yy, *ss.light)
                cnt[rr, c] += 1
    # pixels that see only floor: covered by floor points, as their 8 neighbours
    cov = cnt >= 4
    seen = cov.copy()
    for dr in (-1, 0, 1):
        for dc in (-1, 0, 1):
            seen &= np.roll(np.roll(cov, dr, 0), dc, 1)
    seen[0, :] = seen[-1, :] = False
    seen[:, 0] = seen[:, -1] = False
    assert seen.sum() > 150
    want = acc[seen] / cnt[seen]
    got = img[seen]
    assert abs(got.mean() - want.mean()) < 0.02 * want.mean(), (got.mean(), want.mean())


def _surf_as_scene(ss):
    """A volume scene with the same single camera, for pixel_coords."""
    return synth.Scene(name="cam", n=(1, 1, 1), voxel=1.0, beta_cloud=np.zeros((1, 1, 1), np.float32),
                       cameras=[ss.camera])


def test_surface_adam_first_step_and_projection():
    """Adam's first step moves each coordinate of u = (kappa, gamma / s) by
    exactly lr against the sign of its gradient (the bias-corrected moments
    are g and g^2), i.e. gamma by lr * s; kappa stops at 1 and gamma at 0
    (the ranges of Eq. phong)."""
    th, m, v = O.surf_adam_step([0.5, 30.0], np.zeros(2), np.zeros(2), [3.0, -1e-4], 1, 0.05, 50.0, eps=0.0)
    assert np.allclose(th, [0.45, 32.5], rtol=0, atol=1e-12)
    th, _, _ = O.surf_adam_step([0.98, 1.0], np.zeros(2), np.zeros(2), [-2.0, 7.0], 1, 0.05, 50.0, eps=0.0)
    assert th[0] == 1.0 and th[1] == 0.0



def test_surface_adam_decayed_step_from_zero_moments():
    """At step t = 3 with zero moments and lr_decay = 2 the step size is lr / 2
    and the update is lr/2 (1-b1)/(1-b1^3) / sqrt((1-b2)/(1-b2^3)) per unit
    of u against the gradient's sign (one gradient seen, bias-corrected)."""
    b1, b2 = 0.9, 0.999
    d = 0.5 * 0.04 * ((1 - b1) / (1 - b1 ** 3)) / np.sqrt((1 - b2) / (1 - b2 ** 3))
    th, _, _ = O.surf_adam_step([0.5, 30.0], np.zeros(2), np.zeros(2), [1.0, -1.0], 3, 0.04, 50.0, eps=0.0,
                                lr_decay=2.0)
    assert np.allclose(th, [0.5 - d, 30.0 + 50.0 * d], rtol=0, atol=1e-12)


def test_phong_factor_is_a_power_of_the_lobe_cosine():
    """At kappa = 1 a path's Phong factor is the product of c_k^gamma over its
    Phong vertices (Eq. phong, c clamped at 0), so each event's contribution
    over its diffuse value (kappa = 0) is r(gamma) = P^gamma for one P per
    event: r(2) = r(1)^2, r(3) = r(1)^3 and r(2.5) = r(1)^2.5 (real only for
    r(1) >= 0, which the clamp guarantees).  A wrong exponent or a missing
    clamp breaks these identities."""
    ss = synth.sphere_box(n_paths=1 << 10)
    checked = 0
    for pid in range(0, 1 << 10):
        base = O.surf_render(ss, 0.0, 1.0, first=pid, n=1, n_norm=1)["images"]
        nz = np.nonzero(base)[0]
        if len(nz) != 1:          # one in-view event: its pixel holds exactly its contribution
            continue
        r = [O.surf_render(ss, 1.0, g, first=pid, n=1, n_norm=1)["images"][nz[0]] / base[nz[0]]
             for g in (1.0, 2.0, 3.0, 2.5)]
        if r[0] == 1.0:           # no Phong vertex on this event's path
            continue
        assert abs(r[1] - r[0] ** 2) <= 1e-12 + 1e-9 * r[0] ** 2, (pid, r)
        assert abs(r[2] - r[0] ** 3) <= 1e-12 + 1e-9 * r[0] ** 3, (pid, r)
        assert r[0] >= 0 and abs(r[3] - r[0] ** 2.5) <= 1e-12 + 1e-9 * r[0] ** 2.5, (pid, r)
        checked += 1
    assert checked >= 20


def test_surface_budgets_leave_the_estimate_unchanged():
    """Measuring the float32 budgets of the surface paths (perturbed
    re-sampling) changes neither the images nor the gradient; the budgets
    are non-negative and not all zero."""
    ss = synth.sphere_box(n_paths=1 << 11)
    a = O.surf_render(ss, 0.5, 20.0)
    dl = a["images"] - 0.9 * a["images"].mean()
    b = O.surf_render(ss, 0.5, 20.0, dldi=dl, image_cond=True, grad_cond=True)
    c = O.surf_render(ss, 0.5, 20.0, dldi=dl)
    assert np.array_equal(a["images"], b["images"]) and np.array_equal(b["grad"], c["grad"])
    assert np.all(b["image_cond"] >= 0) and b["image_cond"].max() > 0
    assert np.all(b["grad_cond"] >= 0) and b["grad_cond"].max() > 0
