"""ctypes front end of the FP64 CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the package smoke check and
the benchmark's CPU-baseline leg, never by the library path.  The oracle
shares no code with the CUDA implementation; it takes scene objects by duck
typing (any object with the attributes of a synthetic scene) so that it
imports nothing from the package either.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None
_lock = threading.Lock()

T_NAMES = ["injected", "missed", "escaped", "absorbed", "truncated", "rr_killed",
           "rr_gain", "collisions", "entered", "seg_cross", "shadow_cross", "in_view"]


def build(force: bool = False, plant: str = "") -> str:
    """Compile the oracle into ``oracle/_liboracle.so`` (gcc, OpenMP).

    ``plant`` (tests only) names one of the OR_PLANT_* mistakes of
    oracle.c; that copy is built into ``oracle/_liboracle_<plant>.so`` and
    the real oracle is left alone."""
    path = _LIB_PATH if not plant else os.path.join(_HERE, f"_liboracle_{plant.lower()}.so")
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    if plant:
        cmd.insert(1, f"-DOR_PLANT_{plant.upper()}")
    subprocess.check_call(cmd)
    os.replace(tmp, path)
    return path


class ORScene(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("n_cams", C.c_int32),
        ("max_orders", C.c_int32), ("rr_start", C.c_int32),
        ("epoch", C.c_uint32), ("scene_id", C.c_uint32),
        ("seed", C.c_uint64),
        ("voxel", C.c_double),
        ("origin", C.c_double * 3),
        ("beta_air", C.c_double), ("albedo_cloud", C.c_double),
        ("albedo_air", C.c_double), ("hg_g", C.c_double),
        ("sun", C.c_double * 3),
        ("sun_irradiance", C.c_double),
        ("rr_q", C.c_double),
        ("cams", C.POINTER(C.c_double)),
    ]


class ORSurf(C.Structure):
    _fields_ = [
        ("n_spheres", C.c_int32), ("phong", C.c_int32), ("max_orders", C.c_int32), ("rr_start", C.c_int32),
        ("epoch", C.c_uint32), ("pad", C.c_uint32),
        ("seed", C.c_uint64),
        ("rr_q", C.c_double),
        ("light", C.c_double * 4),
        ("radiance", C.c_double),
        ("spheres", C.POINTER(C.c_double)),
        ("cam", C.c_double * 12),
    ]


_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_u64p = C.POINTER(C.c_uint64)
_u32p = C.POINTER(C.c_uint32)
_i64p = C.POINTER(C.c_int64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


@contextlib.contextmanager
def planted(name: str):
    """Tests only: inside the block, every call goes to a copy of the oracle
    compiled with the planted mistake OR_PLANT_<name> (see oracle.c), so a
    test can show that its pin rejects that mistake."""
    global _lib
    lib()
    with _lock:
        saved = _lib
        _lib = _load(build(plant=name))
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _load(path):
    L = C.CDLL(path)
    L.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.or_fnv1a_words.argtypes = [_u32p, C.c_int]
    L.or_fnv1a_words.restype = C.c_uint64
    L.or_phase_hg.argtypes = [C.c_double, C.c_double]
    L.or_phase_hg.restype = C.c_double
    L.or_phase_rayleigh.argtypes = [C.c_double]
    L.or_phase_rayleigh.restype = C.c_double
    L.or_sample_hg.argtypes = [C.c_double, C.c_double]
    L.or_sample_hg.restype = C.c_double
    L.or_sample_rayleigh.argtypes = [C.c_double]
    L.or_sample_rayleigh.restype = C.c_double
    L.or_rotate.argtypes = [_dp, C.c_double, C.c_double, _dp]
    L.or_onb.argtypes = [_dp, _dp, _dp]
    L.or_pixel_solid_angle.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int]
    L.or_pixel_solid_angle.restype = C.c_double
    L.or_transmittance.argtypes = [C.POINTER(ORScene), _fp, _dp, _dp, C.c_double]
    L.or_transmittance.restype = C.c_double
    L.or_intervals.argtypes = [C.POINTER(ORScene), _dp, _dp, C.c_double, _i64p, _dp, C.c_int]
    L.or_intervals.restype = C.c_int
    L.or_render.argtypes = [C.POINTER(ORScene), _fp, _fp, C.c_uint64, C.c_uint64, C.c_double,
                            _dp, _dp, _dp, _dp, _dp, _dp, _dp, _u64p, C.c_int]
    L.or_render.restype = C.c_int
    L.or_path.argtypes = [C.POINTER(ORScene), _fp, C.c_uint64, _dp, _dp, _i64p, _dp, C.POINTER(C.c_int)]
    L.or_path.restype = C.c_int
    L.or_sun_rect.argtypes = [C.POINTER(ORScene), _dp]
    L.or_single_scatter_quad.argtypes = [C.POINTER(ORScene), _fp, C.c_int, C.c_int, _dp]
    L.or_camera_frame.argtypes = [C.POINTER(ORScene), C.c_int, _dp]
    L.or_surf_render.argtypes = [C.POINTER(ORSurf), C.c_double, C.c_double, C.c_uint64, C.c_uint64,
                                 C.c_double, _dp, _dp, _dp, _dp, _dp, _u64p, _dp, _dp]
    L.or_surf_render.restype = C.c_int
    L.or_space_carve.argtypes = [C.POINTER(ORScene), _dp, C.c_double, C.POINTER(C.c_uint8)]
    L.or_pixel_coords.argtypes = [C.POINTER(ORScene), C.c_int, _dp, _dp]
    L.or_pixel_coords.restype = C.c_int
    L.or_tally_count.restype = C.c_int
    return L


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(t)


class OScene:
    """Keeps the ctypes struct and the arrays it points into alive."""

    def __init__(self, sc, epoch: int = 0, scene_id: int = 0, seed=None):
        # Scene constants are taken at float32 precision, the precision in
        # which the scene is specified to the library under test; the
        # oracle's arithmetic on them is float64.
        f32 = lambda v: float(np.float32(v))
        cams = np.zeros((len(sc.cameras), 12), dtype=np.float64)
        for i, c in enumerate(sc.cameras):
            cams[i, 0:3] = [f32(v) for v in c.pos]
            cams[i, 3:6] = [f32(v) for v in c.look_at]
            cams[i, 6:9] = [f32(v) for v in c.up]
            cams[i, 9] = f32(c.fov_y)
            cams[i, 10] = c.width
            cams[i, 11] = c.height
        self.cams = np.ascontiguousarray(cams)
        s = ORScene()
        s.nx, s.ny, s.nz = (int(k) for k in sc.n)
        s.n_cams = len(sc.cameras)
        s.max_orders = int(sc.max_orders)
        s.rr_start = int(sc.rr_start)
        s.epoch = int(epoch)
        s.scene_id = int(scene_id)
        s.seed = int(sc.seed if seed is None else seed)
        s.voxel = f32(sc.voxel)
        sun = np.array([f32(v) for v in sc.sun_dir], dtype=np.float64)
        sun /= np.linalg.norm(sun)
        for i in range(3):
            s.origin[i] = f32(sc.origin[i])
            s.sun[i] = float(sun[i])
        s.beta_air = f32(sc.beta_air)
        s.albedo_cloud = f32(sc.albedo_cloud)
        s.albedo_air = f32(sc.albedo_air)
        s.hg_g = f32(sc.hg_g)
        s.sun_irradiance = f32(sc.sun_irradiance)
        s.rr_q = f32(sc.rr_q)
        s.cams = self.cams.ctypes.data_as(_dp)
        self.s = s
        self.n_pixels = int(sum(c.width * c.height for c in sc.cameras))
        self.n_voxels = int(sc.n[0] * sc.n[1] * sc.n[2])

    @property
    def ref(self):
        return C.byref(self.s)


def _grid(b):
    return np.ascontiguousarray(np.asarray(b, dtype=np.float32).reshape(-1))


def render(sc, beta_ref, beta_t=None, first: int = 0, n=None, n_norm=None, dldi=None,
           grad_abs: bool = False, grad_cond: bool = False, tallies: bool = False, fingerprints: bool = False,
           threads: int = 1, epoch: int = 0, scene_id: int = 0, seed=None, image_cond: bool = False):
    """Paths [first, first+n) sampled under ``beta_ref``, evaluated under
    ``beta_t`` (default: the same grid).  Returns a dict with ``images``
    (float64, n_pixels), and when asked ``grad``/``grad_abs`` (float64,
    n_voxels), ``tallies`` (dict), ``fingerprints`` (uint64, n) and two error
    budgets for float32 implementations of the same paths:
    ``image_cond`` (per pixel) and ``grad_cond`` (per voxel).  Each is
    measured by perturbation: every path is sampled again four times with
    each computed vertex moved, in a random direction, by a float32 roundoff
    of its coordinates (plus the roundoff of the optical depth accumulated to
    a collision, over beta there), and 4x the largest change over the draws
    of the path's contributions (pixel by pixel) or gradient terms (voxel by
    voxel) is added, together with the roundoff of the crossing times along
    each ray.
    Budgets are large only where the geometry is ill-conditioned: a
    collision in thin air just past cloud edges, a grazing crossing, a
    near-tie of a pixel or voxel decision.
    """
    L = lib()
    os_ = OScene(sc, epoch=epoch, scene_id=scene_id, seed=seed)
    n = int(sc.n_paths if n is None else n)
    n_norm = float(n if n_norm is None else n_norm)
    br = _grid(beta_ref)
    bt = br if beta_t is None else _grid(beta_t)
    img = np.zeros(os_.n_pixels, dtype=np.float64)
    out = {"images": img}
    ic = np.zeros(os_.n_pixels, dtype=np.float64) if image_cond else None
    if ic is not None:
        out["image_cond"] = ic
    g = ga = gc = dl = None
    if dldi is not None:
        dl = np.ascontiguousarray(np.asarray(dldi, dtype=np.float64).reshape(-1))
        g = np.zeros(os_.n_voxels, dtype=np.float64)
        out["grad"] = g
        if grad_abs:
            ga = np.zeros(os_.n_voxels, dtype=np.float64)
            out["grad_abs"] = ga
        if grad_cond:
            gc = np.zeros(os_.n_voxels, dtype=np.float64)
            out["grad_cond"] = gc
    tal = np.zeros(L.or_tally_count(), dtype=np.float64) if tallies else None
    fp = np.zeros(n, dtype=np.uint64) if fingerprints else None
    rc = L.or_render(os_.ref, _ptr(br, _fp), _ptr(bt, _fp), C.c_uint64(first), C.c_uint64(n),
                     C.c_double(n_norm), _ptr(img, _dp), _ptr(ic, _dp), _ptr(dl, _dp), _ptr(g, _dp), _ptr(ga, _dp),
                     _ptr(gc, _dp), _ptr(tal, _dp), _ptr(fp, _u64p), int(threads))
    if rc != 0:
        raise RuntimeError(f"or_render failed ({rc})")
    if tal is not None:
        out["tallies"] = dict(zip(T_NAMES, tal.tolist()))
    if fp is not None:
        out["fingerprints"] = fp
    return out


def path(sc, beta, pid: int, epoch: int = 0, scene_id: int = 0):
    """Vertices of path ``pid``: dict(B, end, x, om, v, l)."""
    L = lib()
    os_ = OScene(sc, epoch=epoch, scene_id=scene_id)
    m = int(sc.max_orders) + 2
    x = np.zeros((m, 3)); om = np.zeros((m, 3)); l = np.zeros(m)
    v = np.zeros(m, dtype=np.int64)
    end = C.c_int(0)
    br = _grid(beta)
    B = L.or_path(os_.ref, _ptr(br, _fp), C.c_uint64(pid), _ptr(x, _dp), _ptr(om, _dp),
                  _ptr(v, _i64p), _ptr(l, _dp), C.byref(end))
    k = max(B, -1) + 1
    return {"B": B, "end": end.value, "x": x[:k], "om": om[:k], "v": v[:k], "l": l[:k]}


def philox(ctr, key):
    L = lib()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    o = np.zeros(4, dtype=np.uint32)
    L.or_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(o, _u32p))
    return o


def fnv1a_words(words):
    w = np.asarray(words, dtype=np.uint32).copy()
    return int(lib().or_fnv1a_words(_ptr(w, _u32p), len(w)))


def phase_hg(g, mu):
    return lib().or_phase_hg(float(g), float(mu))


def phase_rayleigh(mu):
    return lib().or_phase_rayleigh(float(mu))


def sample_hg(g, u):
    return lib().or_sample_hg(float(g), float(u))


def sample_rayleigh(u):
    return lib().or_sample_rayleigh(float(u))


def rotate(d, mu, phi):
    d = np.asarray(d, dtype=np.float64).copy()
    o = np.zeros(3)
    lib().or_rotate(_ptr(d, _dp), float(mu), float(phi), _ptr(o, _dp))
    return o


def onb(n):
    n = np.asarray(n, dtype=np.float64).copy()
    b1 = np.zeros(3); b2 = np.zeros(3)
    lib().or_onb(_ptr(n, _dp), _ptr(b1, _dp), _ptr(b2, _dp))
    return b1, b2


def pixel_solid_angle(tx, ty, W, H, col, row):
    return lib().or_pixel_solid_angle(float(tx), float(ty), int(W), int(H), int(col), int(row))


def transmittance(sc, beta, p, d, tmax):
    os_ = OScene(sc)
    p = np.asarray(p, dtype=np.float64).copy(); d = np.asarray(d, dtype=np.float64).copy()
    b = _grid(beta)
    return lib().or_transmittance(os_.ref, _ptr(b, _fp), _ptr(p, _dp), _ptr(d, _dp), float(tmax))


def intervals(sc, p, d, tmax):
    os_ = OScene(sc)
    cap = int(sum(sc.n)) + 8
    vox = np.zeros(cap, dtype=np.int64); ln = np.zeros(cap)
    p = np.asarray(p, dtype=np.float64).copy(); d = np.asarray(d, dtype=np.float64).copy()
    k = lib().or_intervals(os_.ref, _ptr(p, _dp), _ptr(d, _dp), float(tmax), _ptr(vox, _i64p), _ptr(ln, _dp), cap)
    return vox[:k], ln[:k]


def sun_rect(sc):
    os_ = OScene(sc)
    o = np.zeros(12)
    lib().or_sun_rect(os_.ref, _ptr(o, _dp))
    return {"e1": o[0:3], "e2": o[3:6], "amin": o[6], "amax": o[7], "bmin": o[8], "bmax": o[9],
            "hmin": o[10], "area": o[11]}


def camera_frame(sc, cam):
    os_ = OScene(sc)
    o = np.zeros(14)
    lib().or_camera_frame(os_.ref, int(cam), _ptr(o, _dp))
    return {"C": o[0:3], "F": o[3:6], "R": o[6:9], "U": o[9:12], "tx": o[12], "ty": o[13]}


def single_scatter_quad(sc, beta, sub: int = 8, steps: int = 8):
    os_ = OScene(sc)
    b = _grid(beta)
    img = np.zeros(os_.n_pixels)
    lib().or_single_scatter_quad(os_.ref, _ptr(b, _fp), int(sub), int(steps), _ptr(img, _dp))
    return img


def adam_step(beta, m, v, grad, t, lr, b1=0.9, b2=0.999, eps=1e-8, _plant=""):
    """Adam (Kingma & Ba, Algorithm 1) on beta with projection beta >= 0
    (READING of the paper's "modified Adam": the projection keeps the
    extinction physical); fp64 numpy.  Step t (1-based): moments
    m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, bias-corrected by
    1 - b1^t and 1 - b2^t, step lr m_hat / (sqrt(v_hat) + eps).
    ``_plant`` (tests only) plants a mistake: "no_bias_correction" or
    "no_projection"."""
    beta = np.asarray(beta, dtype=np.float64)
    g = np.asarray(grad, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    if _plant == "no_bias_correction":
        mh, vh = m, v
    beta = beta - lr * mh / (np.sqrt(vh) + eps)
    if _plant != "no_projection":
        beta = np.maximum(beta, 0.0)
    return beta, m, v



def surf_adam_step(theta, m, v, grad, t, lr, gamma_scale, b1=0.9, b2=0.999, eps=1e-8, lr_decay=0.0):
    """Adam on u = (kappa, gamma / gamma_scale) with gradient
    (d/dkappa, gamma_scale d/dgamma) and step size lr / (1 + (t-1)/lr_decay)
    (lr_decay 0: constant), then the projection onto 0 <= kappa <= 1,
    gamma >= 0 that Eq. phong requires; fp64 numpy.
    Returns (theta, m, v), m and v the moments of u."""
    k, gm = np.asarray(theta, dtype=np.float64)
    g = np.asarray(grad, dtype=np.float64)
    if lr_decay > 0:
        lr = lr / (1.0 + (t - 1) / lr_decay)
    u, m, v = adam_step([k, gm / gamma_scale], m, v, [g[0], g[1] * gamma_scale], t, lr, b1, b2, eps)
    return np.array([min(u[0], 1.0), u[1] * gamma_scale]), m, v

def space_carve(sc, images, threshold: float) -> np.ndarray:
    """Photo-hull mask (V uint8, x fastest; 1 = kept) of ``images``
    (camera-major, as render_forward's), see or_space_carve."""
    os_ = OScene(sc)
    im = np.ascontiguousarray(np.asarray(images, dtype=np.float64).reshape(-1))
    mask = np.zeros(os_.n_voxels, dtype=np.uint8)
    lib().or_space_carve(os_.ref, _ptr(im, _dp), float(threshold), mask.ctypes.data_as(C.POINTER(C.c_uint8)))
    return mask


def pixel_coords(sc, cam: int, x):
    """Continuous (column, row) of point x in camera ``cam``, None if behind."""
    os_ = OScene(sc)
    p = np.asarray(x, dtype=np.float64).copy()
    out = np.zeros(2)
    ok = lib().or_pixel_coords(os_.ref, int(cam), _ptr(p, _dp), _ptr(out, _dp))
    return out if ok else None


def _surf(ss, epoch: int = 0, seed=None):
    """ctypes scene; the geometry, light and camera are rounded through
    float32, the precision in which a float32 implementation receives them."""
    f32 = lambda v: float(np.float32(v))
    sph = np.ascontiguousarray(np.asarray(ss.spheres, dtype=np.float32).astype(np.float64).reshape(-1))
    st = ORSurf()
    st.n_spheres = len(sph) // 4
    st.phong = int(ss.phong)
    st.max_orders = int(ss.max_orders)
    st.rr_start = int(ss.rr_start)
    st.epoch = int(epoch)
    st.seed = int(ss.seed if seed is None else seed)
    st.rr_q = f32(ss.rr_q)
    for i in range(4):
        st.light[i] = f32(ss.light[i])
    st.radiance = f32(ss.radiance)
    st.spheres = sph.ctypes.data_as(C.POINTER(C.c_double))
    c = ss.camera
    vals = [f32(v) for v in list(c.pos) + list(c.look_at) + list(c.up) + [c.fov_y]] + [c.width, c.height]
    for i in range(12):
        st.cam[i] = float(vals[i])
    return st, sph


def surf_render(ss, kappa=None, gamma=None, first: int = 0, n=None, n_norm=None, dldi=None, grad_abs: bool = False,
                tallies: bool = False, fingerprints: bool = False, epoch: int = 0, seed=None,
                image_cond: bool = False, grad_cond: bool = False):
    """Reflectometry scene ``ss`` (synth.SurfScene): paths [first, first+n)
    evaluated under (kappa, gamma) (default: the scene's).  Returns images
    (W*H), and when asked grad / grad_abs (2: d loss / d kappa, d gamma),
    tallies (dict), fingerprints, and the float32 budgets image_cond (W*H)
    and grad_cond (2), measured by perturbed re-sampling as render's."""
    L = lib()
    st, keep = _surf(ss, epoch, seed)
    n = int(ss.n_paths if n is None else n)
    n_norm = float(n if n_norm is None else n_norm)
    kappa = float(ss.kappa if kappa is None else kappa)
    gamma = float(ss.gamma if gamma is None else gamma)
    img = np.zeros(ss.n_pixels)
    out = {"images": img}
    dl = g = ga = None
    if dldi is not None:
        dl = np.ascontiguousarray(np.asarray(dldi, dtype=np.float64).reshape(-1))
        g = np.zeros(2)
        out["grad"] = g
        if grad_abs:
            ga = np.zeros(2)
            out["grad_abs"] = ga
    tal = np.zeros(L.or_tally_count(), dtype=np.float64) if tallies else None
    fp = np.zeros(n, dtype=np.uint64) if fingerprints else None
    ic = np.zeros(ss.n_pixels) if image_cond else None
    gc = np.zeros(2) if (grad_cond and dl is not None) else None
    if ic is not None:
        out["image_cond"] = ic
    if gc is not None:
        out["grad_cond"] = gc
    rc = L.or_surf_render(C.byref(st), kappa, gamma, C.c_uint64(first), C.c_uint64(n), n_norm, _ptr(img, _dp),
                          _ptr(dl, _dp), _ptr(g, _dp), _ptr(ga, _dp), _ptr(tal, _dp), _ptr(fp, _u64p),
                          _ptr(ic, _dp), _ptr(gc, _dp))
    if rc != 0:
        raise RuntimeError(f"or_surf_render failed ({rc})")
    if tal is not None:
        out["tallies"] = dict(zip(T_NAMES, tal.tolist()))
    if fp is not None:
        out["fingerprints"] = fp
    return out
