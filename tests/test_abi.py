"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every entry point include/pathrecycle.h declares;
the binding refuses what it cannot run."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pathrecycle.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


def _declared(headers=None):
    src = "\n".join(open(h).read() for h in (headers or HEADERS))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "sizeof")))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("render_forward", "render_grad", "paths_store", "paths_reweight", "paths_free",
              "pt_last_error", "pt_scene_create", "adam_step", "loss_residual"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2110_00085_gb300 import build as B
    path = B.build()
    lib = C.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.pt_version.restype = C.c_char_p
    assert b"sm_103a" in lib.pt_version()


def test_null_arguments_are_rejected_without_a_gpu():
    from paper_2110_00085_gb300 import native as N
    L = N.load()
    assert L.render_forward(None, None, 0, 0, 1.0, 0, 0, None, 0, None, None, None) == 1
    assert b"null" in L.pt_last_error()
    assert L.pt_scene_create(None, None) == 1
    assert L.paths_reweight(None, None, None, 0, None) == 1
    assert L.render_grad(None, None, None, None, 0, None) == 1
    assert L.adam_step(None, None, None, None, None, 0, 0, 0.0, 0.0, 0.0, 0.0, None) == 1
    assert L.pt_inject_error(None, 1, None) == 1
    assert L.pt_check(None, None) == 1
    assert L.paths_cache_token(None) == 0


def test_scene_descriptor_validation_runs_on_host():
    from paper_2110_00085_gb300 import native as N
    L = N.load()
    d = N.PtSceneDesc()
    d.nx = d.ny = d.nz = 4
    d.voxel = 0.0
    h = C.c_void_p()
    assert L.pt_scene_create(C.byref(d), C.byref(h)) == 1
    assert b"voxel" in L.pt_last_error()
    d.voxel = 0.02
    d.n_cams = 0
    assert L.pt_scene_create(C.byref(d), C.byref(h)) == 1
    assert b"n_cams" in L.pt_last_error()


def test_binding_has_no_cpu_fallback():
    """The binding only marshals device tensors; CPU tensors are refused."""
    import torch
    from paper_2110_00085_gb300 import native as N
    with pytest.raises(TypeError):
        N._dev(torch.zeros(4), torch.float32, "beta")


def test_oracle_is_not_imported_by_the_package():
    pkg = os.path.join(ROOT, "paper_2110_00085_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "oracle.c" not in txt, f


def test_probe_arguments_are_checked_without_a_gpu():
    """pt_probe refuses unknown kinds, null buffers and sizes that are not a
    power of two before it launches anything."""
    from paper_2110_00085_gb300 import native as N
    L = N.load()
    assert L.pt_probe(99, None, 0, None, 1, 1, None, None) == 1
    assert L.pt_probe(0, None, 1024, None, 1, 1, None, None) == 1
    assert b"null" in L.pt_last_error()
    assert L.pt_probe(1, C.c_void_p(16), 1000, None, 1, 1, None, None) == 1
    assert b"power of two" in L.pt_last_error()
    assert L.pt_probe(0, C.c_void_p(16), 1024, None, 8, 1, None, None) == 1
    assert b"sink" in L.pt_last_error()


def test_surface_entry_points_reject_null_arguments_without_a_gpu():
    from paper_2110_00085_gb300 import native as N
    L = N._surf_lib()
    assert L.surf_scene_create(None, None) == 1
    assert L.surf_store(None, 0, 1, 1.0, 0, 0, None, None, None, 0, None) == 1
    assert L.surf_reweight(None, 0.5, 10.0, None, 0, None) == 1
    assert L.surf_reweight_dev(None, None, None, 0, None) == 1
    assert L.surf_grad_dev(None, None, None, None, 0, None) == 1
    assert L.surf_adam_step(None, None, None, None, None, 0.1, 0.0, 50.0, 0.9, 0.999, 1e-8, None, 0, None) == 1
    assert b"null" in L.pt_last_error()


def test_header_is_plain_c(tmp_path):
    """include/pathrecycle.h and include/pt_probes.h are C headers: they
    compile as C11 with warnings as errors (no C++ or CUDA types in the
    boundary)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "t.c"
    src.write_text('#include "pathrecycle.h"\n#include "pt_probes.h"\n'
                   'int main(void) { pt_scene* s = 0; (void)s; return PT_OK + PT_PROBE_GATHER_F32; }\n')
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), "-c",
                        str(src), "-o", str(tmp_path / "t.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
