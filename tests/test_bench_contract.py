"""The benchmark's reference arm (the oracle on the host cores) prints one JSON
line with the keys of the benchmark contract; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line(ora):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in j, key
    assert j["impl"] == "reference" and j["n_gpus"] == 1 and j["steps"] == 1
    assert j["value"] > 0 and j["higher_is_better"] is True
    assert j["config"]["workload"] == "batch96_s8p3_19g_x32"
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"] and cb["sample"]
    e = j["e2e"]
    assert e["value"] == j["value"] and e["unit"] == j["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_roofline_fields_on_synthetic_stats():
    """The roofline object's arithmetic, without a GPU: issue-rate roofline of the sweep and the
    HBM fractions beside it follow from the step statistics and the measured constants."""
    sys.path.insert(0, ROOT)
    import bench
    stats = [{"updates": 6.6e11, "sweep_ms": 2250.0, "reduce_ms": 990.0, "sweep_launches": 17000}]
    peaks = {"hbm_gbs": 6500.0, "sm_max_mhz": 2032.0}
    r = bench.roofline(stats, 3500.0, 1, 16, 10, True, peaks, "of measured", 148)
    ups = 6.6e11 / 2.25
    assert r["bound"] == "alu" and r["unit"] == "Ginst/s"
    assert abs(r["peak"] - 4 * 148 * 2032e6 / 1e9) < 1e-9
    m = bench.measured("k_sweep_batch (Q input)")
    assert m is not None, "the profiled sweep source changed: re-measure and update MEASURED"
    assert abs(r["achieved"] - m["inst_per_update"] * ups / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    h = r["hbm"]
    assert abs(h["algorithmic_bytes_per_update"] - 33 * 4 / 80) < 1e-12
    assert abs(h["frac_algorithmic"] - ups * 1.65 / 1e9 / 6500.0) < 1e-12
    assert h["sweep_design_bytes_per_update"] == 8.4
    assert bench.measured("k_moments_q") is not None
    assert 0 < h["iteration_frac_dram_measured"] < 1
