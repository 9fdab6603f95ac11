"""bench.py's JSON line (needs a GPU): one line with the keys and units the
benchmark contract fixes, on a reduced run (small map, few steps, no tracking
or serving legs, a short CPU-baseline sample)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_prints_the_contract_line():
    cmd = [sys.executable, "bench.py", "--n", "200000", "--steps", "5", "--warmup", "3", "--tracking-frames", "0",
           "--serving-requests", "0", "--no-bucket", "--cpu-seconds", "2", "--cpu-seconds-one-core", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [x for x in r.stdout.strip().splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "clocks", "e2e", "gpu_launches", "roofline", "cpu_baseline"):
        assert k in line, k
    assert line["unit"] == "Mpix/s" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 5 and line["warmup"] == 3 and line["n_gpus"] == 1 and line["scaling"] == "weak"
    assert line["gpu_launches"] > 0 and "workload" in line["config"]
    roof = line["roofline"]
    assert roof["bound"] in ("hbm", "alu", "tensor") and roof["achieved"] > 0 and roof["peak"] > 0
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-3
    step = line["roofline_step"]
    assert 0 < step["frac"] <= 1.5 and 0 < step["hbm_frac"] <= 1.5
    assert abs(step["floor_ms"] - sum(v["floor_ms"] for v in line["roofline_per_kernel"].values())) < 1e-3
    work = line["work"]
    assert 0 < work["blend_evaluations_blended"] <= work["blend_evaluations"]
    assert work["blend_evaluations_blended"] + work["blend_evaluations_skipped"] == work["blend_evaluations"]
    e2e = line["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1 and cb["one_core"]["cores"] == 1
    assert "sm_mhz" in line["clocks"] and "reasons" in line["clocks"]
