"""Build libpathrecycle.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked with nvcc into a
shared library next to this file.  No CMake, no torch extension machinery:
the library has a plain C ABI (include/pathrecycle.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpathrecycle.so")
BUILD_DIR = os.path.join(HERE, "_build")
SOURCES = ["pt_sample.cu", "pt_paths.cu", "pt_events.cu", "pt_batch.cu", "pt_api.cu", "pt_static.cu",
           "pt_surf.cu", "pt_probes.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found (CUDA 13 toolkit required)")
    return p


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    inc = os.path.join(HERE, "..", "include")
    files.extend(os.path.join(inc, f) for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    files.append(os.path.abspath(__file__))
    return files


def source_stamp() -> str:
    """SHA-1 (16 hex digits) of the library's sources and header: identifies
    the build whose kernels a cached tuning choice was timed on."""
    import hashlib
    h = hashlib.sha1()
    for f in sorted(_deps()):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(f, "rb") as fh:
                h.update(os.path.basename(f).encode())
                h.update(fh.read())
    return h.hexdigest()[:16]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    objs = [o for o, _ in results]
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        for _, log in results:
            print(log)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
