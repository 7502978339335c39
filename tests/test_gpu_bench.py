"""bench.py's JSON line on a GB300, at a small path budget in a fresh
process: every key of the line is present and consistent with the others
(value from the step time, the roofline fraction from its achieved rate and
peak, the DRAM traffic from the committed ncu record while the kernels
match it), and the CPU oracle's leg reports its sample."""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_bench_line_keys_and_consistency():
    n = 1 << 16
    r = subprocess.run([sys.executable, "bench.py", "--paths", str(n), "--steps", "3", "--warmup", "3",
                        "--no-calibration", "--cpu-seconds", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks",
              "resample", "kernels_ms"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3 and d["config"]["n_paths"] == n
    assert d["value"] == pytest.approx(n / (d["ms_per_step"] * 1e-3), rel=1e-9)
    roof = d["roofline"]
    assert roof["bound"] in ("l2", "hbm", "alu", "tensor")
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"], rel=1e-9)
    import bench
    if bench.profiled_traffic("render_grad", n) is not None and roof["kernel"].startswith("render_grad"):
        assert roof["traffic"] == pytest.approx(bench.profiled_traffic("render_grad", n), rel=1e-9)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and "paths" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] == 8
    # every step launches the library's kernels: reweight, residual, gradient, Adam (+ store every N_r)
    assert d["gpu_launches"] >= 3 * 7
    assert d["clocks"]["samples"] >= 0 and "reasons" in d["clocks"]
