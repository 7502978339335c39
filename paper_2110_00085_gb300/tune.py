"""A small autotuner for the batched persistent launches.

The batched launches have two launch-shape knobs: the register variant
(the compiler's allocation, or one capped so that 10 blocks of 128 threads
fit on an SM, trading a few spills for more resident warps) and the
schedule: the per-scene sequence of single-scene launches (blocks_per_sm
-1), grouped (one block per tile, 0) or persistent with a number of
resident blocks per SM (tiles are fixed at 128 paths / events).
``tune_blocks`` times one reweight + gradient pass of a bound batch for each
candidate shape with CUDA events, keeps the fastest, and caches the choice in
a JSON file keyed by the GPU name and the batch's shape (grid sizes,
cameras, paths per scene), so later runs skip the timing.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

CACHE_ENV = "PT_TUNE_CACHE"


def _cache_path() -> str:
    return os.environ.get(CACHE_ENV, os.path.join(os.path.expanduser("~"), ".cache", "pathrecycle", "tune.json"))


def batch_key(scenes, n_paths) -> str:
    """GPU name, library build (a choice timed on other kernels is not
    reused) and batch shape."""
    from . import build as _build
    sig = [(tuple(int(k) for k in sc.spec.n), len(sc.spec.cameras), int(n)) for sc, n in zip(scenes, n_paths)]
    name = torch.cuda.get_device_name()
    return name + ":" + _build.source_stamp() + ":" + hashlib.sha1(repr(sig).encode()).hexdigest()[:16]


def shapes(batch, blocks=(2, 4, 6, 8)):
    """Candidate launch shapes (reg_cap, blocks_per_sm): the per-scene
    sequence (-1), and for each register variant the grouped schedule (0)
    and the persistent one at the listed block counts below its occupancy
    limit and at the limit."""
    out = [(0, -1)]
    for rc in (0, 1):
        lim = batch.launch_limit(rc)
        out.append((rc, 0))
        for b in sorted(set([x for x in blocks if x < lim] + [lim])):
            out.append((rc, b))
    return out


def tune_blocks(batch, scenes, n_paths, candidates=None, reps: int = 2, use_cache: bool = True):
    """Pick the launch shape (register variant, resident blocks per SM) for
    ``batch`` (a bound native.Batch); returns ((reg_cap, blocks), timings)."""
    key = batch_key(scenes, n_paths)
    path = _cache_path()
    table = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                table = json.load(f)
        except Exception:
            table = {}
    if use_cache and key in table and "reg_cap" in table[key]:
        best = (int(table[key]["reg_cap"]), int(table[key]["blocks_per_sm"]))
        batch.set_launch(*best)
        return best, table[key].get("all")
    cands = list(candidates) if candidates is not None else shapes(batch)
    timings = {}
    for c in cands:
        batch.set_launch(*c)
        batch.reweight(cache=True)
        batch.grad(cache=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            batch.reweight(cache=True)
            batch.grad(cache=True)
        e1.record()
        torch.cuda.synchronize()
        timings[c] = e0.elapsed_time(e1) / reps
    best = min(timings, key=timings.get)
    batch.set_launch(*best)
    named = {f"{rc}:{b}": ms for (rc, b), ms in timings.items()}
    if use_cache:
        table[key] = {"reg_cap": best[0], "blocks_per_sm": best[1], "ms": timings[best], "all": named}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, path)
    return best, named
