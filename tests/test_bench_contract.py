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


def test_headline_line_is_compact(capsys):
    """emit() prints the detail sections first and a headline under 2,000
    characters last, even when the detail is large (CPU only: a synthetic
    result of the full shape)."""
    sys.path.insert(0, ROOT)
    import bench
    case = {"family": "Q", "p": 8, "form": "helmholtz", "ms": 14.3, "dofs_per_s": 9.4e9, "gops_fp64_alg": 346.0}
    out = {"metric": bench.METRIC, "value": 1.2e10, "unit": "DoF/s", "n_gpus": 1, "steps": 20, "warmup": 5,
           "ms_per_step": 200.0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": bench.arm_dtype("tf32x3"), "data": "synthetic",
           "config": {"workload": "w" * 200, "precision": "tf32x3", "families": "Q,DQ", "degrees": "1,2,3,4,5,6,7,8",
                      "l2": "flushed", "parallelism": "1 GPU"},
           "gpu_launches": 4320, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 90, "reasons": []},
           "roofline": {"bound": "alu", "kernel": "k", "achieved": 350.0, "peak": 629.3, "unit": "G FP64 op/s",
                        "frac": 0.556, "traffic": 123456789, "note": "n" * 500},
           "per_case": [case] * 48,
           "arms": {a: {"value": 1e10, "ms_per_step": 200.0, "per_case": [case] * 48}
                    for a in ("tf32x3", "fp64", "tf32x3:stored", "fp64:stored")},
           "speedup_vs_fp64": 3.0,
           "err_vs_oracle": {"per_case": [{"family": "Q", "p": 1, "form": "mass", "tf32x3": 1e-6}] * 48,
                             "max": {"tf32x3": 4e-6, "fp64": 1e-15}, "sample": "s" * 150},
           "e2e": {"value": 1.1e10, "unit": "DoF/s", "h2d_bytes_per_step": 10 ** 9, "d2h_bytes_per_step": 10 ** 9,
                   "note": "x"},
           "extras": {"e%d" % i: {"rows": [case] * 40} for i in range(10)},
           "cpu_baseline": {"value": 3e6, "unit": "DoF/s", "cores": 16, "kind": "oracle",
                            "sample": "oracle per-cell assembly timed on 1000 cells; " + "z" * 400}}
    bench.emit(out)
    lines = capsys.readouterr().out.strip().splitlines()
    last = lines[-1]
    assert len(last) < 2000, len(last)
    h = json.loads(last)
    for k in ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "dtype", "config", "roofline",
              "cpu_baseline", "e2e", "fp64_value", "speedup_vs_fp64", "max_rel_err_vs_oracle", "clocks",
              "gpu_launches"):
        assert k in h, k
    assert h["fp64_value"] == 1e10 and h["max_rel_err_vs_oracle"]["tf32x3"] == 4e-6
    assert all(json.loads(l)["detail"] for l in lines[:-1])
    assert len(lines) == 1 + 4 + 10  # per_case, arms, err_vs_oracle, roofline_note; ten extras (no probes here)
