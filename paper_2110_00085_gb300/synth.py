"""Seeded synthetic scenes: extinction fields, cameras, sun, path budgets.

This module only *generates inputs*.  It holds none of the method's
arithmetic (no sampling, no transmittance, no phase function, no estimator):
the CUDA library and the CPU oracle both consume what it returns, and neither
imports the other.

Scene conventions (shared by every consumer):

* grid of ``n = (nx, ny, nz)`` cubic voxels of side ``voxel`` km, box corner at
  ``origin`` (0, 0, 0), ``z`` up; the extinction array is float32 with ``x``
  fastest, i.e. numpy shape ``(nz, ny, nx)`` in C order;
* the medium has two particle types (Sec. 4.4 of the paper): cloud droplets
  with unknown extinction ``beta_cloud[v]``, albedo ``albedo_cloud`` and a
  Henyey-Greenstein phase function of asymmetry ``hg_g``; air with a known
  uniform extinction ``beta_air``, albedo ``albedo_air`` and a Rayleigh phase
  function;
* a directional sun: ``sun_dir`` is the unit *propagation* direction of its
  parallel rays and ``sun_irradiance`` the irradiance on a plane normal to
  them (Sec. 6.1 uses the sun with parallel rays);
* perspective pinhole cameras on a 60 degree arc in the x-z plane, aimed at
  the box centre, ``up`` = +y, square pixels, field of view fitted to the
  box's bounding sphere;
* path budget ``n_paths``, Philox key ``seed``, at most ``max_orders``
  scattering events, Russian roulette after event ``rr_start`` with survival
  probability ``rr_q``.

The five workloads follow the sizes of the paper's scenes (Table 1: 1e4 to
1e6 voxels, optical densities up to 127 /km, nine cameras, 76-200 px).  None
of the paper's data (LES clouds, the smoke plume) is available, so seeded
Gaussian blobs and value noise stand in for them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Camera:
    pos: tuple
    look_at: tuple
    up: tuple
    fov_y: float  # full vertical field of view, radians
    width: int
    height: int


@dataclasses.dataclass
class Scene:
    name: str
    n: tuple                      # (nx, ny, nz)
    voxel: float                  # km
    beta_cloud: np.ndarray        # float32, shape (nz, ny, nx)
    beta_air: float = 0.0
    albedo_cloud: float = 0.99
    albedo_air: float = 1.0
    hg_g: float = 0.85
    sun_dir: tuple = (0.5, 0.0, -math.sqrt(3.0) / 2.0)
    sun_irradiance: float = 1.0
    cameras: List[Camera] = dataclasses.field(default_factory=list)
    max_orders: int = 10
    rr_start: int = 5
    rr_q: float = 0.8
    n_paths: int = 1 << 18
    seed: int = 1234
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def n_voxels(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def n_pixels(self) -> int:
        return int(sum(c.width * c.height for c in self.cameras))

    @property
    def box_size(self) -> tuple:
        return tuple(float(k) * self.voxel for k in self.n)

    def replace(self, **kw) -> "Scene":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------
# extinction fields
# ----------------------------------------------------------------------------

def _centres(n: int) -> np.ndarray:
    """Voxel-centre coordinates in units of the box side (0..1)."""
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def gaussian_blobs(n: int, n_blobs: int, peak: float, rng: np.random.Generator) -> np.ndarray:
    """Sum of isotropic Gaussian blobs on an n^3 grid, scaled to ``peak``.

    Centres ~ U[0.25, 0.75]^3 (box units), sigma ~ U[1/10, 1/6], amplitude
    ~ U[0.5, 1]; the sum is rescaled so the largest voxel-centre value equals
    ``peak`` (1/km).
    """
    c = _centres(n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    field = np.zeros((n, n, n), dtype=np.float64)
    for _ in range(n_blobs):
        cx, cy, cz = rng.uniform(0.25, 0.75, size=3)
        sig = rng.uniform(1.0 / 10.0, 1.0 / 6.0)
        amp = rng.uniform(0.5, 1.0)
        r2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
        field += amp * np.exp(-0.5 * r2 / (sig * sig))
    field *= peak / field.max()
    return field.astype(np.float32)


def _value_noise_octave(n: int, cells: int, rng: np.random.Generator) -> np.ndarray:
    """Trilinear value noise: U[0,1) lattice of ``cells`` cells per side."""
    lat = rng.uniform(0.0, 1.0, size=(cells + 1, cells + 1, cells + 1))
    g = _centres(n) * cells
    i0 = np.minimum(np.floor(g).astype(np.int64), cells - 1)
    f = g - i0
    # separable trilinear interpolation, axis order (z, y, x)
    def lerp_axis(a, axis):
        lo = np.take(a, i0, axis=axis)
        hi = np.take(a, i0 + 1, axis=axis)
        shape = [1, 1, 1]
        shape[axis] = n
        w = f.reshape(shape)
        return lo * (1.0 - w) + hi * w
    out = lerp_axis(lat, 0)
    out = lerp_axis(out, 1)
    out = lerp_axis(out, 2)
    return out


def value_noise(n: int, cells: List[int], amps: List[float], rng: np.random.Generator) -> np.ndarray:
    """Multi-octave value noise, min-max normalised to [0, 1]."""
    acc = np.zeros((n, n, n), dtype=np.float64)
    for c, a in zip(cells, amps):
        acc += a * _value_noise_octave(n, c, rng)
    acc -= acc.min()
    acc /= max(acc.max(), 1e-300)
    return acc


def thresholded_cloud(noise: np.ndarray, peak: float, thresh: float = 0.5) -> np.ndarray:
    """beta = peak * clamp((noise - t) / (1 - t), 0, 1), max rescaled to peak."""
    b = np.clip((noise - thresh) / (1.0 - thresh), 0.0, 1.0)
    m = b.max()
    if m > 0:
        b *= peak / m
    return b.astype(np.float32)


def cumulus_field(n: int, peak: float, rng: np.random.Generator) -> np.ndarray:
    """5-octave fractal value noise times a vertical profile, thresholded.

    The profile confines cloud to 20%..80% of the box height with a cosine
    taper; the product is thresholded at 0.5 and scaled to ``peak``.
    """
    cells = [4, 8, 16, 32, 64]
    amps = [1.0, 0.5, 0.25, 0.125, 0.0625]
    noise = value_noise(n, cells, amps, rng)
    zc = _centres(n)
    prof = np.where((zc > 0.2) & (zc < 0.8),
                    0.5 - 0.5 * np.cos(2.0 * np.pi * (zc - 0.2) / 0.6), 0.0)
    noise = noise * (0.4 + 0.6 * prof[:, None, None]) * (prof[:, None, None] > 0)
    noise -= noise.min()
    noise /= max(noise.max(), 1e-300)
    return thresholded_cloud(noise, peak, 0.45)


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

def arc_cameras(n_cams: int, box: tuple, width: int, height: int,
                span_deg: float = 30.0, dist_factor: float = 2.0) -> List[Camera]:
    """``n_cams`` cameras on an arc in the x-z plane, view zeniths evenly
    spaced over [-span, +span] degrees, at distance ``dist_factor`` x the
    largest box side from the box centre, aimed at the centre, up = +y.  The
    vertical field of view is fitted to the box's bounding sphere."""
    L = max(box)
    cx, cy, cz = (0.5 * box[0], 0.5 * box[1], 0.5 * box[2])
    R = dist_factor * L
    half_diag = 0.5 * math.sqrt(box[0] ** 2 + box[1] ** 2 + box[2] ** 2)
    fov_y = 2.0 * math.asin(min(half_diag / R, 0.999))
    cams = []
    for i in range(n_cams):
        zen = 0.0 if n_cams == 1 else math.radians(-span_deg + 2.0 * span_deg * i / (n_cams - 1))
        pos = (cx + R * math.sin(zen), cy, cz + R * math.cos(zen))
        cams.append(Camera(pos=pos, look_at=(cx, cy, cz), up=(0.0, 1.0, 0.0),
                           fov_y=fov_y, width=width, height=height))
    return cams


def sun_from_zenith(zenith_deg: float, azimuth_deg: float = 0.0) -> tuple:
    """Unit propagation direction of sun rays for a given solar zenith."""
    th = math.radians(zenith_deg)
    ph = math.radians(azimuth_deg)
    return (math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), -math.cos(th))


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def config(k: int, n_paths: Optional[int] = None) -> Scene:
    """Workload ``k`` (1..5); ``n_paths`` overrides the path budget."""
    if k == 1:
        rng = np.random.default_rng(1)
        n = 32
        beta = gaussian_blobs(n, 3, 20.0, rng)
        sc = Scene(name="blobs32", n=(n, n, n), voxel=0.02, beta_cloud=beta,
                   cameras=arc_cameras(9, (n * 0.02,) * 3, 32, 32),
                   n_paths=1 << 18, seed=1234)
    elif k == 2:
        rng = np.random.default_rng(2)
        n = 64
        beta = gaussian_blobs(n, 8, 20.0, rng)
        sc = Scene(name="blobs64_air", n=(n, n, n), voxel=0.02, beta_cloud=beta,
                   beta_air=0.01, albedo_air=1.0,
                   cameras=arc_cameras(9, (n * 0.02,) * 3, 64, 64),
                   n_paths=1 << 22, seed=1234)
    elif k == 3:
        rng = np.random.default_rng(4)
        n = 128
        noise = value_noise(n, [4, 8, 16], [1.0, 0.5, 0.25], rng)
        beta = thresholded_cloud(noise, 60.0, 0.5)
        sc = Scene(name="noise128", n=(n, n, n), voxel=0.02, beta_cloud=beta,
                   cameras=arc_cameras(15, (n * 0.02,) * 3, 128, 128),
                   n_paths=1 << 24, seed=1234)
    elif k == 5:
        rng = np.random.default_rng(6)
        n = 256
        beta = cumulus_field(n, 80.0, rng)
        sc = Scene(name="cumulus256_air", n=(n, n, n), voxel=0.01, beta_cloud=beta,
                   beta_air=0.01, albedo_air=1.0,
                   cameras=arc_cameras(21, (n * 0.01,) * 3, 256, 256),
                   n_paths=1 << 28, seed=1234)
    else:
        raise ValueError(f"workload {k}: use batch_config() for the batched workload")
    if n_paths is not None:
        sc = sc.replace(n_paths=int(n_paths))
    return sc


def batch_config(seed: int = 5, n_scenes: int = 16, path_scale: int = 0) -> List[Scene]:
    """Batched workload: ``n_scenes`` clouds of uneven sizes.

    Grid side from {32, 48, 64, 96, 128}, 5..21 cameras at 64x64, 2^(20..23)
    paths per scene (each exponent lowered by ``path_scale``), blob and noise
    recipes alternating.
    """
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_scenes):
        n = int(rng.choice([32, 48, 64, 96, 128]))
        n_cams = int(rng.integers(5, 22))
        k = int(rng.integers(20, 24)) - path_scale
        if s % 2 == 0:
            beta = gaussian_blobs(n, int(rng.integers(2, 9)), 20.0, rng)
        else:
            beta = thresholded_cloud(value_noise(n, [4, 8, 16], [1.0, 0.5, 0.25], rng), 40.0, 0.5)
        out.append(Scene(name=f"batch{s}_{n}", n=(n, n, n), voxel=0.02, beta_cloud=beta,
                         cameras=arc_cameras(n_cams, (n * 0.02,) * 3, 64, 64),
                         n_paths=1 << max(k, 4), seed=1234 + s))
    return out


def small_scene(n: int = 8, n_cams: int = 3, px: int = 8, peak: float = 20.0,
                seed: int = 7, beta_air: float = 0.0, n_paths: int = 1 << 12) -> Scene:
    """A tiny blob scene for brute-force and finite-difference checks."""
    rng = np.random.default_rng(seed)
    beta = gaussian_blobs(n, 2, peak, rng)
    return Scene(name=f"tiny{n}", n=(n, n, n), voxel=0.02, beta_cloud=beta,
                 beta_air=beta_air, cameras=arc_cameras(n_cams, (n * 0.02,) * 3, px, px),
                 n_paths=n_paths, seed=seed)


@dataclasses.dataclass
class SurfScene:
    """A closed unit box for the reflectometry workload (Sec. 6): diffuse
    walls, a square Lambertian emitter in the ceiling (z = 1), diffuse
    spheres and one sphere (index ``phong``) with the Phong BRDF."""
    spheres: np.ndarray           # (n, 4): centre, radius
    phong: int
    light: tuple                  # emitter x0, x1, y0, y1 on z = 1
    radiance: float
    camera: Camera
    kappa: float = 0.7
    gamma: float = 50.0
    max_orders: int = 10
    rr_start: int = 5
    rr_q: float = 0.8
    n_paths: int = 1 << 20
    seed: int = 1234

    def replace(self, **kw) -> "SurfScene":
        return dataclasses.replace(self, **kw)

    @property
    def n_pixels(self) -> int:
        return self.camera.width * self.camera.height


def sphere_box(seed: int = 7, n_small: int = 14, px: int = 60, kappa: float = 0.7, gamma: float = 50.0,
               n_paths: int = 1 << 20) -> SurfScene:
    """Seeded stand-in for the reflectometry scene: a Phong sphere (radius
    0.2) at the centre of the unit box, ``n_small`` diffuse spheres (radius
    0.04-0.08) placed by rejection (inside the box, apart from each other
    and from the large sphere, away from the camera), the emitter on the
    ceiling square [0.35, 0.65]^2 and one camera of ``px`` x ``px`` pixels
    just inside the front wall, looking at the centre."""
    rng = np.random.default_rng(seed)
    sph = [(0.5, 0.5, 0.5, 0.2)]
    while len(sph) < 1 + n_small:
        r = float(rng.uniform(0.04, 0.08))
        c = rng.uniform(r + 0.02, 1.0 - r - 0.02, size=3)
        if c[1] < 0.25:
            continue
        if all(np.linalg.norm(c - np.array(s[:3])) > s[3] + r + 0.02 for s in sph):
            sph.append((float(c[0]), float(c[1]), float(c[2]), r))
    cam = Camera(pos=(0.5, 0.02, 0.45), look_at=(0.5, 0.6, 0.5), up=(0.0, 0.0, 1.0),
                 fov_y=math.radians(70.0), width=px, height=px)
    return SurfScene(spheres=np.array(sph, dtype=np.float64), phong=0, light=(0.35, 0.65, 0.35, 0.65),
                     radiance=1.0, camera=cam, kappa=kappa, gamma=gamma, n_paths=n_paths, seed=seed)
