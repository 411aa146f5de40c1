"""The benchmark's reference arm (the oracle timed on the host) on CPU: it
times the workload its line names, so its `config` is the one the GPU arm
prints for the same `--n`, and its cpu_baseline states the mesh it ran."""
import io
import json
import os
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Args:
    gpus = 1
    steps = 2
    warmup = 3
    n = 16


def test_reference_line_times_its_own_config(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(_Args()) == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["config"] == bench.vortex_config(16, "single GPU")
    assert line["config"]["nv"] == 256 and line["cpu_baseline"]["nv"] == 256
    assert line["steps"] == 2 and line["warmup"] == 3
    assert "2 SSP-RK3 step(s)" in line["cpu_baseline"]["sample"] and "256-vertex" in line["cpu_baseline"]["sample"]
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
