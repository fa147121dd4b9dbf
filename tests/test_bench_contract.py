"""The benchmark's reference arm (the CPU oracle timed on the host cores) and its
JSON line, on CPU: one line with the contract's keys from rank 0, nothing from
the other ranks, and the op counters the roofline divides by."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--steps", "1", "--warmup", "3", "--degrees", "1,2", "--families", "Q,DQ", "--dims", "4,4,4",
         "--cpu-seconds", "1"]


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    r = run_bench(["--impl", "reference"] + SMALL)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in out, k
    assert out["value"] > 0 and out["unit"] == "DoF/s" and out["higher_is_better"] is True
    assert out["steps"] == 1 and out["warmup"] == 3
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"] and cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "4x4x4" in out["config"]["workload"]


def test_reference_arm_other_ranks_print_nothing():
    r = run_bench(["--impl", "reference", "--gpus", "2"] + SMALL,
                  {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_op_counters():
    sys.path.insert(0, ROOT)
    import bench
    for fam in ("Q", "DQ"):
        prev = 0
        for p in range(1, 9):
            for form in ("mass", "laplace", "helmholtz"):
                assert bench.fp64_ops_per_cell(fam, p, form) > 0
                assert bench.mixed_fp64_ops_per_cell(fam, p, form) > 0
            # the FP64 kernel's count grows with the degree; the split kernel does less FP64 work
            cur = bench.fp64_ops_per_cell(fam, p, "laplace")
            assert cur > prev
            assert bench.mixed_fp64_ops_per_cell(fam, p, "laplace") < cur
            prev = cur
    assert bench.launches_per_action("Q") == 8 and bench.launches_per_action("DQ") == 1
    assert bench.job_value(1000, 4, 10.0) == pytest.approx(400000.0)
