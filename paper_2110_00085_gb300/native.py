"""Thin ctypes binding of libpathrecycle.so (C ABI in include/pathrecycle.h).

Argument marshalling only: torch tensors provide device memory and the
current CUDA stream; every step of the computation runs in the library's
kernels.  There is no CPU fallback: if the library is missing or no GPU is
present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np
import torch

from . import build as _build

PT_ACCUMULATE = 1
PT_CACHE = 2
PT_SORT = 4
PT_ASYNC = 8
TALLY_NAMES = ["injected", "missed", "escaped", "absorbed", "truncated", "rr_killed",
               "rr_gain", "collisions", "entered", "seg_cross", "shadow_cross", "in_view"]
TALLY_COUNT = len(TALLY_NAMES)
MAX_ORDERS = 15

_lib = None
_lock = threading.Lock()


class PtCamera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("fov_y", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class PtSceneDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("voxel", C.c_float), ("origin", C.c_float * 3),
                ("beta_air", C.c_float), ("albedo_cloud", C.c_float), ("albedo_air", C.c_float),
                ("hg_g", C.c_float), ("sun_dir", C.c_float * 3), ("sun_irradiance", C.c_float),
                ("n_cams", C.c_int32), ("cams", C.POINTER(PtCamera)),
                ("max_orders", C.c_int32), ("rr_start", C.c_int32), ("rr_q", C.c_float),
                ("scene_id", C.c_uint32)]


class PtPathsInfo(C.Structure):
    _fields_ = [("n_paths", C.c_uint64), ("n_stored", C.c_uint64), ("n_records", C.c_uint64),
                ("bucket", C.c_uint64 * (MAX_ORDERS + 1)), ("bytes_device", C.c_uint64)]


_vp = C.c_void_p
_u64 = C.c_uint64
_u32 = C.c_uint32


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libpathrecycle.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(path)
        L.pt_scene_create.argtypes = [C.POINTER(PtSceneDesc), C.POINTER(_vp)]
        L.pt_scene_free.argtypes = [_vp]
        L.pt_scene_pixels.argtypes = [_vp]
        L.pt_scene_pixels.restype = C.c_int64
        L.render_forward.argtypes = [_vp, _vp, _u64, _u64, C.c_double, _u64, _u32, _vp, _u32, _vp, _vp, _vp]
        L.paths_store.argtypes = [_vp, _vp, _u64, _u64, C.c_double, _u64, _u32, C.POINTER(_vp), _vp, _u32,
                                  _vp, _vp, _vp]
        L.paths_reweight.argtypes = [_vp, _vp, _vp, _u32, _vp]
        L.render_grad.argtypes = [_vp, _vp, _vp, _vp, _u32, _vp]
        L.paths_free.argtypes = [_vp]
        L.paths_cache_token.argtypes = [_vp]
        L.paths_drop_cache.argtypes = [_vp]
        L.paths_cache_token.restype = _u64
        L.paths_info.argtypes = [_vp, C.POINTER(PtPathsInfo), _vp]
        L.adam_step.argtypes = [_vp, _vp, _vp, _vp, _vp, C.c_int64, C.c_int32, C.c_float, C.c_float, C.c_float,
                                C.c_float, _vp]
        L.loss_residual.argtypes = [_vp, _vp, C.c_int64, _vp, _vp, _vp]
        L.space_carve.argtypes = [_vp, _vp, C.c_double, _vp, _vp]
        L.pt_inject_error.argtypes = [_vp, C.c_int, _vp]
        L.adam_step_counted.argtypes = [_vp, _vp, _vp, _vp, _vp, C.c_int64, _vp, _vp, C.c_float, C.c_float, C.c_float,
                                        C.c_float, _vp]
        L.pt_check.argtypes = [_vp, _vp]
        L.render_forward_static.argtypes = [C.POINTER(PtSceneDesc), _vp, _u64, _u64, C.c_double, _u64, _u32,
                                            _vp, _u32, _vp]
        L.batch_create.argtypes = [C.POINTER(_vp), C.c_int, C.POINTER(_vp)]
        L.batch_bind.argtypes = [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), _vp]
        L.batch_reweight.argtypes = [_vp, _u32, _vp]
        L.batch_grad.argtypes = [_vp, _u32, _vp]
        L.batch_set_launch.argtypes = [_vp, C.c_int, C.c_int]
        L.batch_launch_limits.argtypes = [_vp, C.c_int, C.POINTER(C.c_int)]
        L.batch_free.argtypes = [_vp]
        L.pt_probe.argtypes = [C.c_int, _vp, C.c_int64, _vp, C.c_int64, C.c_int, _vp, _vp]
        L.pt_last_error.restype = C.c_char_p
        L.pt_version.restype = C.c_char_p
        _lib = L
        return L


def _check(rc: int, what: str):
    if rc != 0:
        msg = load().pt_last_error().decode(errors="replace")
        raise RuntimeError(f"{what} failed (status {rc}): {msg}")


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev(t: torch.Tensor, dtype, what: str, numel: Optional[int] = None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what}: expected {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _opt(t, dtype, what, numel=None):
    return None if t is None else _dev(t, dtype, what, numel)


class Scene:
    """A scene on the current CUDA device (cameras, pixel solid angles, sun).

    ``sc`` is any object with the attributes of a synthetic scene (grid
    dims, voxel, medium constants, sun, cameras, termination settings).
    """

    def __init__(self, sc, scene_id: int = 0):
        L = load()
        cams = (PtCamera * len(sc.cameras))()
        for i, c in enumerate(sc.cameras):
            cams[i].pos[:] = [float(v) for v in c.pos]
            cams[i].look_at[:] = [float(v) for v in c.look_at]
            cams[i].up[:] = [float(v) for v in c.up]
            cams[i].fov_y = float(c.fov_y)
            cams[i].width = int(c.width)
            cams[i].height = int(c.height)
        d = PtSceneDesc()
        d.nx, d.ny, d.nz = (int(k) for k in sc.n)
        d.voxel = float(sc.voxel)
        d.origin[:] = [float(v) for v in sc.origin]
        d.beta_air = float(sc.beta_air)
        d.albedo_cloud = float(sc.albedo_cloud)
        d.albedo_air = float(sc.albedo_air)
        d.hg_g = float(sc.hg_g)
        d.sun_dir[:] = [float(v) for v in sc.sun_dir]
        d.sun_irradiance = float(sc.sun_irradiance)
        d.n_cams = len(sc.cameras)
        d.cams = cams
        d.max_orders = int(sc.max_orders)
        d.rr_start = int(sc.rr_start)
        d.rr_q = float(sc.rr_q)
        d.scene_id = int(scene_id)
        h = _vp()
        _check(L.pt_scene_create(C.byref(d), C.byref(h)), "pt_scene_create")
        self._h = h
        self.spec = sc
        self.n_pixels = int(L.pt_scene_pixels(h))
        self.n_voxels = int(sc.n[0] * sc.n[1] * sc.n[2])
        self.device = torch.cuda.current_device()

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().pt_scene_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_images(self) -> torch.Tensor:
        return torch.zeros(self.n_pixels, dtype=torch.float64, device="cuda")

    def check(self, stream=None):
        _check(load().pt_check(self._h, _vp(_stream(stream))), "pt_check")

    def inject_error(self, bits: int, stream=None):
        """Test hook: record invariant-violation bits as a kernel would."""
        _check(load().pt_inject_error(self._h, int(bits), _vp(_stream(stream))), "pt_inject_error")

    def space_carve(self, images: torch.Tensor, threshold: float, mask: Optional[torch.Tensor] = None,
                    stream=None) -> torch.Tensor:
        """Photo-hull mask (uint8, 1 = kept) of the cloud seen in ``images``."""
        if mask is None:
            mask = torch.empty(self.n_voxels, dtype=torch.uint8, device="cuda")
        rc = load().space_carve(self._h, _dev(images, torch.float64, "images", self.n_pixels), float(threshold),
                                _dev(mask, torch.uint8, "mask", self.n_voxels), _vp(_stream(stream)))
        _check(rc, "space_carve")
        return mask

    def render_forward(self, beta: torch.Tensor, n_paths: int, seed: int, first: int = 0, n_norm=None,
                       epoch: int = 0, images: Optional[torch.Tensor] = None, accumulate: bool = False,
                       tallies: Optional[torch.Tensor] = None, fingerprints: Optional[torch.Tensor] = None,
                       stream=None) -> torch.Tensor:
        if images is None:
            images = self.new_images()
        n_norm = float(n_paths if n_norm is None else n_norm)
        rc = load().render_forward(self._h, _dev(beta, torch.float32, "beta", self.n_voxels), first, n_paths,
                                   n_norm, seed, epoch, _dev(images, torch.float64, "images", self.n_pixels),
                                   PT_ACCUMULATE if accumulate else 0,
                                   _opt(tallies, torch.float64, "tallies", TALLY_COUNT),
                                   _opt(fingerprints, torch.int64, "fingerprints", n_paths),
                                   _vp(_stream(stream)))
        _check(rc, "render_forward")
        return images


class Paths:
    """Stored, size-sorted light paths (a ``pt_paths`` handle)."""

    def __init__(self, scene: Scene):
        self.scene = scene
        self._h = _vp()

    def store(self, beta: torch.Tensor, n_paths: int, seed: int, first: int = 0, n_norm=None, epoch: int = 0,
              images_ref: Optional[torch.Tensor] = None, accumulate: bool = False,
              tallies: Optional[torch.Tensor] = None, fingerprints: Optional[torch.Tensor] = None, stream=None,
              asynchronous: bool = False):
        """``asynchronous``: PT_ASYNC (no stream synchronisation on a handle an
        earlier store has sized; a set that does not fit, or an invalid
        grid, is reported by Scene.check())."""
        n_norm = float(n_paths if n_norm is None else n_norm)
        sc = self.scene
        flags = (PT_ACCUMULATE if accumulate else 0) | (PT_ASYNC if asynchronous else 0)
        rc = load().paths_store(sc.handle, _dev(beta, torch.float32, "beta", sc.n_voxels), first, n_paths, n_norm,
                                seed, epoch, C.byref(self._h),
                                _opt(images_ref, torch.float64, "images_ref", sc.n_pixels),
                                flags,
                                _opt(tallies, torch.float64, "tallies", TALLY_COUNT),
                                _opt(fingerprints, torch.int64, "fingerprints", n_paths),
                                _vp(_stream(stream)))
        _check(rc, "paths_store")
        return self

    def reweight(self, beta_t: torch.Tensor, images: Optional[torch.Tensor] = None, cache: bool = False,
                 accumulate: bool = False, stream=None) -> torch.Tensor:
        sc = self.scene
        if images is None:
            images = sc.new_images()
        flags = (PT_CACHE if cache else 0) | (PT_ACCUMULATE if accumulate else 0)
        rc = load().paths_reweight(self._h, _dev(beta_t, torch.float32, "beta_t", sc.n_voxels),
                                   _dev(images, torch.float64, "images", sc.n_pixels), flags,
                                   _vp(_stream(stream)))
        _check(rc, "paths_reweight")
        return images

    def grad(self, beta_t: torch.Tensor, dldi: torch.Tensor, grad: Optional[torch.Tensor] = None,
             cache: bool = False, accumulate: bool = False, stream=None) -> torch.Tensor:
        sc = self.scene
        if grad is None:
            grad = torch.zeros(sc.n_voxels, dtype=torch.float64, device="cuda")
        flags = (PT_CACHE if cache else 0) | (PT_ACCUMULATE if accumulate else 0)
        rc = load().render_grad(self._h, _dev(beta_t, torch.float32, "beta_t", sc.n_voxels),
                                _dev(dldi, torch.float64, "dL_dI", sc.n_pixels),
                                _dev(grad, torch.float64, "grad", sc.n_voxels), flags, _vp(_stream(stream)))
        _check(rc, "render_grad")
        return grad

    def drop_cache(self):
        """Free the contribution cache (the next cached reweight allocates it again)."""
        _check(load().paths_drop_cache(self._h), "paths_drop_cache")

    def cache_token(self) -> int:
        """Which cache-writing reweight the contribution cache holds (0: none)."""
        return int(load().paths_cache_token(self._h))

    def info(self, stream=None) -> dict:
        inf = PtPathsInfo()
        _check(load().paths_info(self._h, C.byref(inf), _vp(_stream(stream))), "paths_info")
        return {"n_paths": inf.n_paths, "n_stored": inf.n_stored, "n_records": inf.n_records,
                "bucket": list(inf.bucket), "bytes_device": inf.bytes_device}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().paths_free(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adam_step(beta, m, v, grad, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8,
              mask=None, stream=None):
    """Adam + projection beta >= 0; ``mask`` (uint8, optional): voxels with 0 stay."""
    n = beta.numel()
    rc = load().adam_step(_dev(beta, torch.float32, "beta"), _dev(m, torch.float32, "m", n),
                          _dev(v, torch.float32, "v", n), _dev(grad, torch.float64, "grad", n),
                          _opt(mask, torch.uint8, "mask", n), n, int(t),
                          float(lr), float(b1), float(b2), float(eps), _vp(_stream(stream)))
    _check(rc, "adam_step")


def adam_step_counted(beta, m, v, grad, step, scratch, lr: float, b1: float = 0.9, b2: float = 0.999,
                      eps: float = 1e-8, mask=None, stream=None):
    """Adam with the step number in device memory (``step``: int32[1])."""
    n = beta.numel()
    rc = load().adam_step_counted(_dev(beta, torch.float32, "beta"), _dev(m, torch.float32, "m", n),
                                  _dev(v, torch.float32, "v", n), _dev(grad, torch.float64, "grad", n),
                                  _opt(mask, torch.uint8, "mask", n), n,
                                  _dev(step, torch.int32, "step", 1), _dev(scratch, torch.float32, "scratch", 2),
                                  float(lr), float(b1), float(b2), float(eps), _vp(_stream(stream)))
    _check(rc, "adam_step_counted")


def loss_residual(images, gt, dldi=None, loss=None, stream=None):
    n = images.numel()
    if dldi is None:
        dldi = torch.empty_like(images)
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float64, device=images.device)
    rc = load().loss_residual(_dev(images, torch.float64, "images"), _dev(gt, torch.float64, "gt", n), n,
                              _dev(dldi, torch.float64, "dL_dI", n), _dev(loss, torch.float64, "loss", 1),
                              _vp(_stream(stream)))
    _check(rc, "loss_residual")
    return dldi, loss


def scene_desc(sc, scene_id: int = 0):
    """(pt_scene_desc, camera array) for a synthetic scene; keep both alive
    while the description is in use."""
    cams = (PtCamera * len(sc.cameras))()
    for i, c in enumerate(sc.cameras):
        cams[i].pos[:] = [float(v) for v in c.pos]
        cams[i].look_at[:] = [float(v) for v in c.look_at]
        cams[i].up[:] = [float(v) for v in c.up]
        cams[i].fov_y = float(c.fov_y)
        cams[i].width = int(c.width)
        cams[i].height = int(c.height)
    d = PtSceneDesc()
    d.nx, d.ny, d.nz = (int(k) for k in sc.n)
    d.voxel = float(sc.voxel)
    d.origin[:] = [float(v) for v in sc.origin]
    d.beta_air = float(sc.beta_air)
    d.albedo_cloud = float(sc.albedo_cloud)
    d.albedo_air = float(sc.albedo_air)
    d.hg_g = float(sc.hg_g)
    d.sun_dir[:] = [float(v) for v in sc.sun_dir]
    d.sun_irradiance = float(sc.sun_irradiance)
    d.n_cams = len(sc.cameras)
    d.cams = cams
    d.max_orders = int(sc.max_orders)
    d.rr_start = int(sc.rr_start)
    d.rr_q = float(sc.rr_q)
    d.scene_id = int(scene_id)
    return d, cams


def render_forward_static(sc, beta: torch.Tensor, n_paths: int, seed: int, first: int = 0, n_norm=None,
                          epoch: int = 0, images: Optional[torch.Tensor] = None, accumulate: bool = False,
                          scene_id: int = 0, stream=None) -> torch.Tensor:
    """render_forward without a pt_scene, for callers that cannot allocate
    device memory (the library keeps the scene tables in a fixed device
    array; at most 16 cameras and 2^18 pixels)."""
    d, cams = scene_desc(sc, scene_id)
    n_pix = int(sum(c.width * c.height for c in sc.cameras))
    n_vox = int(sc.n[0] * sc.n[1] * sc.n[2])
    if images is None:
        images = torch.zeros(n_pix, dtype=torch.float64, device=beta.device)
    n_norm = float(n_paths if n_norm is None else n_norm)
    rc = load().render_forward_static(C.byref(d), _dev(beta, torch.float32, "beta", n_vox), first, n_paths, n_norm,
                                      seed, epoch, _dev(images, torch.float64, "images", n_pix),
                                      PT_ACCUMULATE if accumulate else 0, _vp(_stream(stream)))
    _check(rc, "render_forward_static")
    return images


(PROBE_GATHER_F32, PROBE_RED_F64, PROBE_RED_F64_WARP, PROBE_RED_F64_SAME, PROBE_RED_F32, PROBE_COPY,
 PROBE_SHARED_F32, PROBE_SHARED_F32_RUN4, PROBE_SHARED_U32, PROBE_SHARED_F64) = range(10)


def probe(kind: int, buf: torch.Tensor, iters: int = 0, blocks: int = 0, src: Optional[torch.Tensor] = None,
          sink: Optional[torch.Tensor] = None, stream=None):
    """One memory-rate probe (include/pt_probes.h) on ``buf``: random gathers
    or reductions (``iters`` per thread, ``blocks`` x 256 threads) or a
    streaming copy ``src`` -> ``buf`` (16-byte elements)."""
    if not isinstance(buf, torch.Tensor) or not buf.is_cuda or not buf.is_contiguous():
        raise TypeError("probe: buf must be a contiguous CUDA tensor")
    esz = 16 if kind == PROBE_COPY else (8 if kind in (PROBE_RED_F64, PROBE_RED_F64_WARP, PROBE_RED_F64_SAME)
                                          else 4)   # shared probes: one float32 per thread
    n = buf.numel() * buf.element_size() // esz
    sp = None
    if src is not None:
        if not src.is_cuda or src.numel() * src.element_size() < n * esz:
            raise ValueError("probe: src must be a CUDA tensor at least as large as buf")
        sp = src.data_ptr()
    rc = load().pt_probe(int(kind), buf.data_ptr(), n, sp, int(iters), int(blocks),
                         None if sink is None else _dev(sink, torch.float32, "sink"), _vp(_stream(stream)))
    _check(rc, "pt_probe")


class Batch:
    """Several stored-path handles run as one persistent launch per pass."""

    def __init__(self, paths_list):
        self.paths = list(paths_list)
        arr = (_vp * len(self.paths))(*[p._h.value for p in self.paths])
        h = _vp()
        _check(load().batch_create(arr, len(self.paths), C.byref(h)), "batch_create")
        self._h = h
        self._bound = None
        self.shape = (0, self.launch_limit(0))   # the library's default launch shape

    def bind(self, betas, images, dldis, grads, stream=None):
        n = len(self.paths)
        def ptrs(ts, dtype, what, sizes):
            return (_vp * n)(*[_dev(t, dtype, what, k) for t, k in zip(ts, sizes)])
        vox = [p.scene.n_voxels for p in self.paths]
        pix = [p.scene.n_pixels for p in self.paths]
        args = (ptrs(betas, torch.float32, "beta_t", vox), ptrs(images, torch.float64, "images", pix),
                ptrs(dldis, torch.float64, "dL_dI", pix), ptrs(grads, torch.float64, "grad", vox))
        _check(load().batch_bind(self._h, *args, _vp(_stream(stream))), "batch_bind")
        self._bound = (list(betas), list(images), list(dldis), list(grads))   # keep the tensors alive

    def reweight(self, cache: bool = True, accumulate: bool = False, stream=None):
        flags = (PT_CACHE if cache else 0) | (PT_ACCUMULATE if accumulate else 0)
        _check(load().batch_reweight(self._h, flags, _vp(_stream(stream))), "batch_reweight")

    def grad(self, cache: bool = True, accumulate: bool = False, stream=None):
        flags = (PT_CACHE if cache else 0) | (PT_ACCUMULATE if accumulate else 0)
        _check(load().batch_grad(self._h, flags, _vp(_stream(stream))), "batch_grad")

    def set_launch(self, reg_cap: int, blocks_per_sm: int):
        """Launch shape: register variant (0 compiler's, 1 capped for 10
        blocks per SM) and resident blocks per SM of the persistent
        schedule, or 0 for the grouped schedule (one block per tile), or -1
        for the per-scene sequence."""
        _check(load().batch_set_launch(self._h, int(reg_cap), int(blocks_per_sm)), "batch_set_launch")
        self.shape = (int(reg_cap), int(blocks_per_sm))

    def kernels_per_step(self) -> tuple:
        """Kernels of this library launched by (reweight, grad) in the
        current shape: per-scene sequence = 3 + 2 per scene, grouped = 3 + 2
        per group of up to 64 scenes, persistent = tile offsets + 3 and tile
        offsets + 2."""
        if self.shape[1] == -1:
            return 3 * len(self.paths), 2 * len(self.paths)
        if self.shape[1] == 0:
            g = (len(self.paths) + 63) // 64
            return 3 * g, 2 * g
        return 4, 3

    def launch_limit(self, reg_cap: int) -> int:
        """Occupancy limit (resident blocks per SM) of register variant reg_cap."""
        m = C.c_int(0)
        _check(load().batch_launch_limits(self._h, int(reg_cap), C.byref(m)), "batch_launch_limits")
        return m.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().batch_free(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ reflectometry --
class PtSurfDesc(C.Structure):
    _fields_ = [("n_spheres", C.c_int32), ("spheres", C.POINTER(C.c_float)), ("phong", C.c_int32),
                ("light", C.c_float * 4), ("radiance", C.c_float), ("camera", PtCamera),
                ("max_orders", C.c_int32), ("rr_start", C.c_int32), ("rr_q", C.c_float)]


_surf_bound = False


def _surf_lib():
    global _surf_bound
    L = load()
    if not _surf_bound:
        L.surf_scene_create.argtypes = [C.POINTER(PtSurfDesc), C.POINTER(_vp)]
        L.surf_scene_free.argtypes = [_vp]
        L.surf_scene_pixels.argtypes = [_vp]
        L.surf_scene_pixels.restype = C.c_int64
        L.surf_store.argtypes = [_vp, C.c_uint64, C.c_uint64, C.c_double, C.c_uint64, C.c_uint32, C.POINTER(_vp),
                                 _vp, _vp, C.c_uint32, _vp]
        L.surf_reweight.argtypes = [_vp, C.c_double, C.c_double, _vp, C.c_uint32, _vp]
        L.surf_grad.argtypes = [_vp, C.c_double, C.c_double, _vp, _vp, C.c_uint32, _vp]
        L.surf_reweight_dev.argtypes = [_vp, _vp, _vp, C.c_uint32, _vp]
        L.surf_grad_dev.argtypes = [_vp, _vp, _vp, _vp, C.c_uint32, _vp]
        L.surf_adam_step.argtypes = [_vp, _vp, _vp, _vp, _vp, C.c_float, C.c_float, C.c_float, C.c_float,
                                     C.c_float, C.c_float, _vp, C.c_int32, _vp]
        L.surf_paths_events.argtypes = [_vp, C.POINTER(C.c_uint64)]
        L.surf_paths_free.argtypes = [_vp]
        _surf_bound = True
    return L


class SurfScene:
    """Device scene of the reflectometry workload (synth.SurfScene)."""

    def __init__(self, ss):
        L = _surf_lib()
        self.spec = ss
        self._sph = np.ascontiguousarray(np.asarray(ss.spheres, dtype=np.float32).reshape(-1))
        d = PtSurfDesc()
        d.n_spheres = len(self._sph) // 4
        d.spheres = self._sph.ctypes.data_as(C.POINTER(C.c_float))
        d.phong = int(ss.phong)
        d.light[:] = [float(v) for v in ss.light]
        d.radiance = float(ss.radiance)
        c = ss.camera
        d.camera.pos[:] = [float(v) for v in c.pos]
        d.camera.look_at[:] = [float(v) for v in c.look_at]
        d.camera.up[:] = [float(v) for v in c.up]
        d.camera.fov_y = float(c.fov_y)
        d.camera.width = int(c.width)
        d.camera.height = int(c.height)
        d.max_orders = int(ss.max_orders)
        d.rr_start = int(ss.rr_start)
        d.rr_q = float(ss.rr_q)
        h = _vp()
        _check(L.surf_scene_create(C.byref(d), C.byref(h)), "surf_scene_create")
        self._h = h
        self.n_pixels = int(L.surf_scene_pixels(h))

    def new_images(self) -> torch.Tensor:
        return torch.zeros(self.n_pixels, dtype=torch.float64, device="cuda")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _surf_lib().surf_scene_free(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SurfPaths:
    """Stored light paths of a SurfScene, re-evaluated under BRDF parameters."""

    def __init__(self, scene: SurfScene):
        self.scene = scene
        self._h = _vp()

    def store(self, n_paths: int, seed: int, first: int = 0, n_norm=None, epoch: int = 0, tallies=None,
              fingerprints=None, sort: bool = True, stream=None):
        """Trace light paths [first, first + n_paths); ``sort`` orders the kept
        events by pixel (worth it when the paths are re-evaluated repeatedly)."""
        n_norm = float(n_paths if n_norm is None else n_norm)
        rc = _surf_lib().surf_store(self.scene._h, first, n_paths, n_norm, seed, epoch, C.byref(self._h),
                                    _opt(tallies, torch.float64, "tallies", TALLY_COUNT),
                                    _opt(fingerprints, torch.int64, "fingerprints", n_paths),
                                    PT_SORT if sort else 0, _vp(_stream(stream)))
        _check(rc, "surf_store")
        return self

    def reweight(self, kappa: float, gamma: float, images=None, accumulate: bool = False, stream=None):
        if images is None:
            images = self.scene.new_images()
        rc = _surf_lib().surf_reweight(self._h, float(kappa), float(gamma),
                                       _dev(images, torch.float64, "images", self.scene.n_pixels),
                                       PT_ACCUMULATE if accumulate else 0, _vp(_stream(stream)))
        _check(rc, "surf_reweight")
        return images

    def grad(self, kappa: float, gamma: float, dldi, grad=None, accumulate: bool = False, stream=None):
        if grad is None:
            grad = torch.zeros(2, dtype=torch.float64, device="cuda")
        rc = _surf_lib().surf_grad(self._h, float(kappa), float(gamma),
                                   _dev(dldi, torch.float64, "dL_dI", self.scene.n_pixels),
                                   _dev(grad, torch.float64, "grad", 2), PT_ACCUMULATE if accumulate else 0,
                                   _vp(_stream(stream)))
        _check(rc, "surf_grad")
        return grad

    def reweight_dev(self, theta, images=None, accumulate: bool = False, stream=None):
        """reweight with (kappa, gamma) read from ``theta`` (device float32[2])."""
        if images is None:
            images = self.scene.new_images()
        rc = _surf_lib().surf_reweight_dev(self._h, _dev(theta, torch.float32, "theta", 2),
                                           _dev(images, torch.float64, "images", self.scene.n_pixels),
                                           PT_ACCUMULATE if accumulate else 0, _vp(_stream(stream)))
        _check(rc, "surf_reweight_dev")
        return images

    def grad_dev(self, theta, dldi, grad=None, accumulate: bool = False, stream=None):
        if grad is None:
            grad = torch.zeros(2, dtype=torch.float64, device="cuda")
        rc = _surf_lib().surf_grad_dev(self._h, _dev(theta, torch.float32, "theta", 2),
                                       _dev(dldi, torch.float64, "dL_dI", self.scene.n_pixels),
                                       _dev(grad, torch.float64, "grad", 2), PT_ACCUMULATE if accumulate else 0,
                                       _vp(_stream(stream)))
        _check(rc, "surf_grad_dev")
        return grad

    def events(self) -> int:
        n = C.c_uint64(0)
        _check(_surf_lib().surf_paths_events(self._h, C.byref(n)), "surf_paths_events")
        return n.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _surf_lib().surf_paths_free(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def surf_adam_step(theta, m, v, grad, step, lr: float, gamma_scale: float, b1: float = 0.9, b2: float = 0.999,
                   eps: float = 1e-8, trace=None, lr_decay: float = 0.0, stream=None):
    """Adam on (kappa, gamma / gamma_scale) with the projection of Eq. phong;
    theta, m, v: device float32[2]; grad: float64[2]; step: int32[1];
    step size lr / (1 + (t - 1) / lr_decay) (lr_decay 0: constant);
    trace (optional float32[2 * T]): (kappa, gamma) after each step."""
    cap = 0 if trace is None else trace.numel() // 2
    rc = _surf_lib().surf_adam_step(_dev(theta, torch.float32, "theta", 2), _dev(m, torch.float32, "m", 2),
                                    _dev(v, torch.float32, "v", 2), _dev(grad, torch.float64, "grad", 2),
                                    _dev(step, torch.int32, "step", 1), float(lr), float(lr_decay),
                                    float(gamma_scale), float(b1),
                                    float(b2), float(eps), _opt(trace, torch.float32, "trace", 2 * cap), cap,
                                    _vp(_stream(stream)))
    _check(rc, "surf_adam_step")
