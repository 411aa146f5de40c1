"""The benchmark's JSON line on a small mesh: one line with the fields its
readers rely on (the metric and its figures, the roofline of the dominant
kernel, the end-to-end figure with the bytes it copies, the clock record,
the launch count) and sane values.  The adjoint and batch sub-objects are
left out here (--skip-legs); their functions run in the GPU tests of their
own workloads."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_fields():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--n", "60", "--steps", "3", "--warmup", "3",
           "--skip-legs", "--no-cpu-baseline"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks", "f64_dw", "fp32"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3 and d["dtype"] == "f64"
    assert d["config"]["nv"] == 3600 and d["config"]["ne"] == 10800
    assert d["value"] > 0 and abs(d["value"] - 3600 * 3 * 3 / (d["ms_per_step"] * 3 / 1e3) / 1e6) < 0.01 * d["value"]
    r = d["roofline"]
    assert r["bound"] == "alu" and 0 < r["frac"] < 1.2 and r["unit"] == "TFLOP/s"
    assert d["e2e"]["h2d_bytes_per_step"] == 3600 * 32 and d["e2e"]["d2h_bytes_per_step"] == 3600 * 32
    assert d["e2e"]["value"] > 0 and len(d["e2e"]["block_values"]) == 3
    assert d["gpu_launches"] == 6 * 3
    assert d["fp32"]["error_vs_f64"]["rho"] < 1e-5 and d["f64_dw"]["residual_vs_f64"] < 1e-12
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
