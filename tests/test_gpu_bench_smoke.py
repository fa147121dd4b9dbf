"""Benchmark smoke runs on the GPU at reduced sizes: `bench.py` exits 0, prints
its detail lines first and the compact headline JSON last, under 2,000
characters, with every key of its contract (roofline, end-to-end rate with the
copied bytes, clocks, launch count, the FP64 arm and the error against the
oracle), values in range."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "gpu_launches", "clocks", "roofline", "e2e")


def run(args):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    last = lines[-1]
    assert len(last) < 2000, len(last)
    out = json.loads(last)
    details = [json.loads(l) for l in lines[:-1] if l.startswith("{")]
    assert all("detail" in d for d in details)
    return out, {d["detail"]: d["data"] for d in details}


def check_headline(out):
    for k in KEYS:
        assert k in out, k
    assert out["value"] > 0 and out["ms_per_step"] > 0 and out["n_gpus"] == 1
    assert out["warmup"] >= 3 and out["higher_is_better"] is True
    rf = out["roofline"]
    assert rf["bound"] == "alu" and rf["unit"] == "G FP64 op/s" and rf["frac"] > 0
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"], abs=1e-4)  # frac is rounded to 4 places
    e2e = out["e2e"]
    assert e2e["value"] > 0 and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] == e2e["h2d_bytes_per_step"]
    assert "sm_mhz" in out["clocks"] and "reasons" in out["clocks"]


def test_bench_smoke_json_line():
    out, det = run(["--steps", "1", "--warmup", "3", "--degrees", "1,2", "--families", "Q,DQ", "--dims", "8,8,8",
                    "--no-extras", "--no-cpu-baseline", "--no-autotune", "--precision", "tf32x3,fp64"])
    check_headline(out)
    assert out["steps"] == 1
    # 12 cases: Q_p actions take 8 colour launches, DQ_p actions one
    assert out["gpu_launches"] == (6 * 8 + 6 * 1) * out["steps"]
    assert "8x8x8" in out["config"]["workload"]
    assert out["dtype"].startswith("tf32x3")
    assert out["fp64_value"] > 0 and out["speedup_vs_fp64"] > 0
    err = out["max_rel_err_vs_oracle"]
    assert err["fp64"] <= 1e-12 and err["tf32x3"] <= 2e-5
    assert len(det["per_case"]) == 12 and len(det["err_vs_oracle"]["per_case"]) == 12


def test_bench_default_output_path_small():
    """The default run's output path (every arm, the other workloads, the CPU
    baseline), with the other workloads shrunk: the last line still parses
    and stays under 2,000 characters."""
    out, det = run(["--steps", "1", "--warmup", "3", "--degrees", "1,2", "--dims", "8,8,8", "--small-extras",
                    "--cpu-seconds", "1", "--no-autotune"])
    check_headline(out)
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1
    assert set(out["max_rel_err_vs_oracle"]) == {"tf32x3", "fp64"}
    assert any(k.startswith("extras.") for k in det)
    assert "arms" in det and "tf32x3:stored" in det["arms"]
    # the precision extra: each precision's sampled error against the oracle
    # (Q_p Laplace and vector Q_p neo-Hookean), within the parity tolerances
    rows = det["extras.precision_64cube"]["rows"]
    assert rows
    for r in rows:
        assert r["fp64_rel_err_vs_oracle_sampled"] <= 1e-12
        assert r["tf32x3_rel_err_vs_oracle_sampled"] <= 2e-5
        assert r["bf16x3_rel_err_vs_oracle_sampled"] <= 2e-3
