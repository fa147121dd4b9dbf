"""Benchmark smoke run on the GPU at a reduced size: `bench.py` exits 0 and
prints one JSON line with every key of its contract (roofline, end-to-end rate
with the copied bytes, clocks, launch count), values in range."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_smoke_json_line():
    args = ["--steps", "1", "--warmup", "3", "--degrees", "1,2", "--families", "Q,DQ", "--dims", "8,8,8",
            "--no-extras", "--no-cpu-baseline", "--no-autotune", "--precision", "tf32x3,fp64"]
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "gpu_launches", "clocks", "roofline", "e2e"):
        assert k in out, k
    assert out["value"] > 0 and out["ms_per_step"] > 0 and out["n_gpus"] == 1
    assert out["steps"] == 1 and out["warmup"] >= 3 and out["higher_is_better"] is True
    # 12 cases: Q_p actions take 8 colour launches, DQ_p actions one
    assert out["gpu_launches"] == (6 * 8 + 6 * 1) * out["steps"]
    rf = out["roofline"]
    assert rf["bound"] == "alu" and rf["unit"] == "G FP64 op/s" and rf["frac"] > 0
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"], abs=1e-4)  # frac is rounded to 4 places
    e2e = out["e2e"]
    assert e2e["value"] > 0 and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] == e2e["h2d_bytes_per_step"]
    assert "sm_mhz" in out["clocks"] and "reasons" in out["clocks"]
    assert "8x8x8" in out["config"]["workload"]
