"""Pins of the oracle's two-particle-type medium (cloud + air) and of its
volumetric Adam step.

The forward estimate with air has three parts that the cloud-only pins do
not reach: the air term of the scattering function at a local estimate, the
choice of the particle type that scatters (which sets the direction pdf),
and the albedo factor of a scattering vertex in the path weight.  Each is
pinned here against mathematics the paper fixes, and each test also plants
the plausible mistake in a copy of the oracle (oracle.c OR_PLANT_*, or the
Adam hook) and checks that the pin rejects it.

Closed forms (Sec. 3.2, the integrated RTE, for a laterally infinite
homogeneous slab lit by a collimated sun of irradiance F0 at cosine mu0 and
seen from above at cosine mu):
  I1 = F0 P(Theta) mu0/(mu0+mu) [1 - exp(-tau (1/mu0 + 1/mu))]
  I2 = (F0/mu) int dOmega' P(Omega'.Omega) P(Omega0.Omega') K(Omega')
with P = f_s / beta = (alb_c beta_c f^c + alb_a beta_a f^a) / (beta_c + beta_a)
the mixed phase function times the mixed albedo (Sec. 3.1) and K the depth
integral of the first-order radiance (derived in _second_order_slab).
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2110_00085_gb300 import synth

G = 0.85


def p_hg(mu, g=G):
    """Henyey-Greenstein phase function (normalised on the sphere)."""
    return (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * mu) ** 1.5)


def p_ray(mu):
    """Rayleigh phase function (normalised on the sphere)."""
    return 3.0 / (16.0 * math.pi) * (1 + mu * mu)


def cdf_hg(mu, g=G):
    return (1 - g * g) / (2 * g) * ((1 + g * g - 2 * g * mu) ** -0.5 - 1 / (1 + g))


def cdf_ray(mu):
    return (mu ** 3 + 3 * mu + 4) / 8


# cloud 6 /km (albedo 0.99, HG) + air 4 /km (albedo 0.5, Rayleigh): albedo_air
# differs from 1 and from the cloud's, so weighting the types by extinction
# instead of by scattering changes every quantity below
BC, BA, ALB_C, ALB_A = 6.0, 4.0, 0.99, 0.5


def _slab(n_paths, max_orders):
    nxy, nz = 64, 2
    beta = np.full((nz, nxy, nxy), BC, np.float32)
    box = (nxy * 0.02, nxy * 0.02, nz * 0.02)
    return synth.Scene(name="slab2", n=(nxy, nxy, nz), voxel=0.02, beta_cloud=beta, beta_air=BA,
                       albedo_cloud=ALB_C, albedo_air=ALB_A, hg_g=G, sun_dir=synth.sun_from_zenith(30.0),
                       cameras=synth.arc_cameras(1, box, 16, 16), max_orders=max_orders, rr_start=5,
                       n_paths=n_paths, seed=4242)


def _f32(x):
    return float(np.float32(x))


def _central_dirs(sc):
    """Propagation directions toward the camera (Omega, z up) at the centres
    of the 8x8 central pixels (which see the slab at least 0.4 km, 16 mean
    free paths, inside its edges), and the pixel indices."""
    f = O.camera_frame(sc, 0)
    out = []
    for row in range(4, 12):
        for col in range(4, 12):
            x = f["tx"] * (-1 + 2 * (col + 0.5) / 16)
            y = f["ty"] * (1 - 2 * (row + 0.5) / 16)
            d = f["F"] + x * f["R"] + y * f["U"]
            d /= np.linalg.norm(d)
            out.append((row * 16 + col, -d))
    return out


def _first_order_slab(sc, om):
    s = np.array(sc.sun_dir)
    mu0, mu = -s[2], om[2]
    tau = (_f32(BC) + _f32(BA)) * 0.04
    return float(_P(float(s @ om))) * mu0 / (mu0 + mu) * (1 - math.exp(-tau * (1 / mu0 + 1 / mu)))


def _second_order_slab(sc, om, n_mu=200, n_phi=256):
    """Second-order radiance leaving the top of the slab along om.

    First-order radiance at optical depth t (from the top) along a
    direction of vertical cosine mu' (m = |mu'|), with P0 = P(Omega0.Omega'):
      downward: F0 P0 mu0/(m - mu0) [exp(-t/m) - exp(-t/mu0)]
      upward:   F0 P0 mu0/(mu0 + m) [exp(-t/mu0) - exp(-tau/mu0 - (tau - t)/m)]
    Scattered once more toward om and attenuated by exp(-t/mu) on the way
    out, its depth integral over [0, tau] is F0 P0 K with, for
    Fi(a) = int_0^tau exp(-a t) dt = (1 - exp(-a tau)) / a,
      downward: K = mu0/(m - mu0) [Fi(1/m + 1/mu) - Fi(1/mu0 + 1/mu)]
      upward:   K = mu0/(mu0 + m) [Fi(1/mu0 + 1/mu) - exp(-tau (1/mu0 + 1/mu)) Fi(1/m - 1/mu)]
    and I2 = (1/mu) int dOmega' P(Omega'.om) P0 K.  Directions: Gauss-Legendre
    in mu' on each hemisphere, the trapezoid rule in azimuth."""
    s = np.array(sc.sun_dir)
    mu0, mu = -s[2], om[2]
    tau = (_f32(BC) + _f32(BA)) * 0.04

    def Fi(a):
        a = np.asarray(a, dtype=np.float64)
        small = np.abs(a) < 1e-9
        return np.where(small, tau, -np.expm1(-a * tau) / np.where(small, 1.0, a))   # a >= 0 or |a tau| small

    x, w = np.polynomial.legendre.leggauss(n_mu)
    m = 0.5 * (x + 1)
    wm = 0.5 * w
    phi = 2 * math.pi * np.arange(n_phi) / n_phi
    wphi = 2 * math.pi / n_phi
    total = 0.0
    for up in (False, True):
        muz = m if up else -m
        st = np.sqrt(1 - muz ** 2)
        d = np.stack([st[:, None] * np.cos(phi)[None, :], st[:, None] * np.sin(phi)[None, :],
                      np.broadcast_to(muz[:, None], (n_mu, n_phi))], axis=-1)
        c_in = d @ s          # Omega0 . Omega'
        c_out = d @ om        # Omega' . Omega
        P_in = _P(c_in)
        P_out = _P(c_out)
        mm = m[:, None]
        if up:
            K = mu0 / (mu0 + mm) * (Fi(1 / mu0 + 1 / mu) - math.exp(-tau * (1 / mu0 + 1 / mu)) * Fi(1 / mm - 1 / mu))
        else:
            K = mu0 / (mm - mu0) * (Fi(1 / mm + 1 / mu) - Fi(1 / mu0 + 1 / mu))
        total += float(np.sum(wm[:, None] * wphi * P_out * P_in * K))
    return total / mu


def _P(mu):
    """f_s / beta of the slab medium: the mixed phase function times the
    mixed albedo (the oracle takes the constants at float32)."""
    bc, ba, ac, aa = _f32(BC), _f32(BA), _f32(ALB_C), _f32(ALB_A)
    return (ac * bc * p_hg(mu) + aa * ba * p_ray(mu)) / (bc + ba)


def _block_images(sc, blocks=16, threads=8):
    n = sc.n_paths // blocks
    return np.array([O.render(sc, sc.beta_cloud, first=b * n, n=n, threads=threads)["images"]
                     for b in range(blocks)])


def _order1_check(n_paths=1 << 20):
    sc = _slab(n_paths, 1)
    ims = _block_images(sc)
    pix = _central_dirs(sc)
    mc = np.array([ims[:, k].mean() for k, _ in pix])
    sd = np.array([ims[:, k].std(ddof=1) / math.sqrt(len(ims)) for k, _ in pix])
    ex = np.array([_first_order_slab(sc, om) for _, om in pix])
    ratio = mc.sum() / ex.sum()
    return ratio, math.sqrt((sd ** 2).sum()) / ex.sum()


def _order2_check(n_paths=1 << 22):
    """Order-2 image (max_orders 2 minus max_orders 1 on the same paths: the
    two runs share every draw up to the first collision's local estimate)
    against the quadrature; returns the ratio of sums and its standard error."""
    i2 = _block_images(_slab(n_paths, 2))
    i1 = _block_images(_slab(n_paths, 1))
    d = i2 - i1
    sc = _slab(n_paths, 2)
    pix = _central_dirs(sc)
    mc = np.array([d[:, k].mean() for k, _ in pix])
    sd = np.array([d[:, k].std(ddof=1) / math.sqrt(len(d)) for k, _ in pix])
    ex = np.array([_second_order_slab(sc, om) for _, om in pix])
    return mc.sum() / ex.sum(), math.sqrt((sd ** 2).sum()) / ex.sum()


def test_slab_quadratures_converge_and_reproduce_the_first_order_closed_form():
    """The quadrature of the second-order radiance is converged (two
    resolutions agree to 1e-3), and its P integrates over the sphere to the
    mixed albedo beta_s / beta (both phase functions normalised, Sec. 3.1)."""
    sc = _slab(1 << 10, 2)
    for _, om in _central_dirs(sc)[:3]:
        a = _second_order_slab(sc, om, 200, 256)
        b = _second_order_slab(sc, om, 400, 512)
        assert abs(a - b) < 1e-3 * abs(b)
        assert a > 0
    x, w = np.polynomial.legendre.leggauss(400)
    tot = 2 * math.pi * float(np.sum(w * _P(x)))
    alb = (_f32(ALB_C) * _f32(BC) + _f32(ALB_A) * _f32(BA)) / (_f32(BC) + _f32(BA))
    assert abs(tot - alb) < 1e-6


def test_two_type_slab_single_scattering():
    """First-order radiance of a cloud + air slab (albedo_air 0.5) equals
    the closed form with the mixed scattering function (1% + 4 sigma); the
    oracle with the air term weighted by extinction (beta_a instead of
    albedo_a beta_a in f_s) fails it."""
    ratio, se = _order1_check()
    assert abs(ratio - 1) < 0.01 + 4 * se, (ratio, se)
    with O.planted("AIR_BY_EXTINCTION"):
        bad, bse = _order1_check(1 << 18)
    assert abs(bad - 1) > 0.2 + 4 * bse, (bad, bse)


def test_two_type_slab_second_order():
    """Second-order radiance of the cloud + air slab (type chosen at the
    first collision, direction from that type's phase function, the vertex
    albedo in the weight) equals the quadrature of the second-order RTE term
    (2% + 4 sigma).  Planted: the direction pdf normalised by extinction
    (drops the vertex albedo) and the type chosen by extinction both fail."""
    ratio, se = _order2_check()
    assert abs(ratio - 1) < 0.02 + 4 * se, (ratio, se)
    for plant in ("DIRECTION_PDF_BY_EXTINCTION", "TYPE_BY_EXTINCTION"):
        with O.planted(plant):
            bad, bse = _order2_check(1 << 20)
        assert abs(bad - 1) > 0.1 + 4 * bse, (plant, bad, bse)


def _first_scatter_cosines(n):
    sc = _slab(n, 3)
    mus = []
    for pid in range(n):
        p = O.path(sc, sc.beta_cloud, pid)
        if p["B"] >= 1 and len(p["om"]) >= 2:
            mus.append(float(np.dot(p["om"][0], p["om"][1])))
    return np.array(mus)


def test_first_scatter_direction_follows_the_mixed_phase_function():
    """At a collision in cloud + air the cosine between incoming and
    outgoing directions is distributed as the mixture of HG and Rayleigh
    with weights albedo_j beta_j / beta_s (the type choice that makes the
    direction pdf f_p): Kolmogorov-Smirnov against the closed-form CDFs,
    and the first two moments (HG: g, (1 + 2g^2)/3; Rayleigh: 0, 2/5).
    The oracle that picks the type by extinction fails both."""
    bc, ba, ac, aa = _f32(BC), _f32(BA), _f32(ALB_C), _f32(ALB_A)
    wc = ac * bc / (ac * bc + aa * ba)

    def cdf(mu):
        return wc * cdf_hg(mu) + (1 - wc) * cdf_ray(mu)

    m1 = wc * G
    m2 = wc * (1 + 2 * G * G) / 3 + (1 - wc) * 0.4
    mus = _first_scatter_cosines(32000)     # about a third of the paths enter and collide
    assert len(mus) > 10000
    assert stats.kstest(mus, cdf).pvalue > 1e-3
    n = len(mus)
    assert abs(mus.mean() - m1) < 4 * mus.std() / math.sqrt(n)
    assert abs((mus ** 2).mean() - m2) < 4 * (mus ** 2).std() / math.sqrt(n)
    with O.planted("TYPE_BY_EXTINCTION"):
        bad = _first_scatter_cosines(32000)
    assert stats.kstest(bad, cdf).pvalue < 1e-6
    assert abs(bad.mean() - m1) > 6 * bad.std() / math.sqrt(len(bad))


# ------------------------------------------------------------- volumetric Adam
def test_adam_first_step_is_the_step_size_along_minus_the_gradient_sign():
    """Kingma & Ba: after one step from zero moments the bias-corrected
    moments are g and g^2, so the step is lr g / (|g| + eps): every voxel
    with |g| >> eps moves by lr against the sign of its gradient, and a zero
    gradient does not move.  Without the bias correction the first step is
    lr (1 - b1) / sqrt(1 - b2) = 3.16 lr, which the pin rejects."""
    beta = np.array([5.0, 5.0, 5.0, 5.0])
    g = np.array([3e-3, -7.0, 0.0, 1e4])
    z = np.zeros(4)
    lr, eps = 0.25, 1e-8
    b, m, v = O.adam_step(beta, z, z, g, 1, lr, eps=eps)
    assert np.allclose(b, beta - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-12)
    assert np.allclose(b, beta - lr * np.sign(g), rtol=0, atol=1e-5 * lr)
    bb, _, _ = O.adam_step(beta, z, z, g, 1, lr, _plant="no_bias_correction")
    assert not np.allclose(bb, beta - lr * np.sign(g), rtol=0, atol=1e-3)


def test_adam_steps_under_a_constant_gradient_are_all_lr():
    """With a constant gradient the bias-corrected moments equal g and g^2
    at every step t (the corrections divide out the geometric sums), so t
    steps move a voxel by exactly t lr."""
    beta = np.array([10.0, 10.0])
    g = np.array([0.5, -2.0])
    m = v = np.zeros(2)
    lr = 0.1
    for t in range(1, 26):
        beta, m, v = O.adam_step(beta, m, v, g, t, lr)
        assert np.allclose(beta, 10.0 - t * lr * np.sign(g), rtol=0, atol=1e-6)
    b2 = np.array([10.0, 10.0]); m2 = v2 = np.zeros(2)
    for t in range(1, 4):
        b2, m2, v2 = O.adam_step(b2, m2, v2, g, t, lr, _plant="no_bias_correction")
    assert not np.allclose(b2, 10.0 - 3 * lr * np.sign(g), rtol=0, atol=1e-3)


def test_adam_second_step_after_the_gradient_vanishes():
    """Gradient g then 0: the second step is lr (b1 / (1 + b1)) / sqrt(b2 /
    (1 + b2)) in the first step's direction (bias-corrected moments
    b1 (1 - b1) g / (1 - b1^2) and b2 (1 - b2) g^2 / (1 - b2^2)); at the
    default b1 = 0.9, b2 = 0.999 that is 0.670058 lr."""
    b1, b2, lr = 0.9, 0.999, 1.0
    beta = np.array([10.0])
    z = np.zeros(1)
    beta, m, v = O.adam_step(beta, z, z, np.array([2.0]), 1, lr)
    beta2, _, _ = O.adam_step(beta, m, v, np.array([0.0]), 2, lr)
    step = float(beta[0] - beta2[0])
    expect = lr * (b1 / (1 + b1)) / math.sqrt(b2 / (1 + b2))
    assert abs(expect - 0.6700583) < 1e-6
    assert abs(step - expect) < 1e-7


def test_adam_projection_keeps_extinction_non_negative():
    """The projection beta >= 0: a voxel asked to step below zero stops at
    zero, one far from zero steps freely; the oracle without the projection
    goes negative."""
    beta = np.array([0.05, 3.0])
    g = np.array([1.0, 1.0])
    z = np.zeros(2)
    b, _, _ = O.adam_step(beta, z, z, g, 1, 0.2)
    assert b[0] == 0.0 and abs(b[1] - 2.8) < 1e-8
    bb, _, _ = O.adam_step(beta, z, z, g, 1, 0.2, _plant="no_projection")
    assert bb[0] < 0
