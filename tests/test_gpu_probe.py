"""The throughput probes the benchmark reports beside its roofline: each probe
runs, counts its work, and lands in a plausible range of GB300's nominal
rates (an FP64 FMA rate above the FP64 pipe's nominal 2 per clock per SM at
the maximum clock would mean the work is miscounted)."""
import pytest

pytestmark = pytest.mark.gpu


def test_probes_run_and_are_plausible(gpu):
    sfx, torch, ctx = gpu
    import bench
    r = bench.probe_rates(sfx, torch, target_ms=5.0)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    nominal_dfma = nsm * 2 * 2.07  # G FMA/s
    assert 0.3 * nominal_dfma < r["dfma"]["rate"] <= 1.05 * nominal_dfma, r
    assert r["ffma"]["rate"] > 10 * r["dfma"]["rate"], r
    assert r["mma_tf32"]["rate"] > 10.0 and r["mma_bf16"]["rate"] > r["mma_tf32"]["rate"] * 0.9, r
    assert r["dmma"]["rate"] > 0.1, r
