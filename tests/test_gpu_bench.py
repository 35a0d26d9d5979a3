"""bench.py's native arm at a small size: the JSON line carries every key of the
benchmark contract (roofline, gather views, clocks, end-to-end, launch count,
the oracle baseline on the host cores), with self-consistent values."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_native_line_contract(tmp_path):
    out = tmp_path / "b.json"
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--particles", "4096", "--keyframes", "4",
           "--steps", "3", "--warmup", "3", "--e2e-steps", "2", "--cpu-particles", "256", "--out", str(out)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = json.loads(out.read_text())
    assert json.loads(r.stdout.strip().splitlines()[-1]) == line
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "gather", "clocks", "gpu_launches", "e2e",
              "cpu_baseline"):
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == 3 and line["warmup"] == 3 and line["scaling"] == "weak"
    assert line["higher_is_better"] is True and line["value"] > 0 and line["vs_baseline"] is None
    assert "workload" in line["config"] and "l2" in line["config"]
    # value = P * N * 3 moves per frame over the mean frame time
    assert abs(line["value"] - 4096 * 2048 * 3 / (line["ms_per_step"] * 1e-3)) <= 1e-6 * line["value"]
    rf = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in rf, k
    assert rf["bound"] == "alu" and rf["unit"] == "TFLOP/s" and 0 < rf["frac"] < 1.2
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    e2e = line["e2e"]
    assert e2e["unit"] == line["unit"] and e2e["value"] > 0
    assert e2e["h2d_bytes_per_step"] == 2048 * 12 and e2e["d2h_bytes_per_step"] > 0
    assert line["gpu_launches"] == 16 * 3          # 16 kernel launches per frame, 3 timed frames
    ck = line["clocks"]
    assert "sm_mhz" in ck and "sm_max_mhz" in ck and isinstance(ck["reasons"], list)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and cb["unit"] == line["unit"]
