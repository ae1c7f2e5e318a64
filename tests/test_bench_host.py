"""Host-side pieces of bench.py that need no GPU: the workload description of the JSON line, the
measured-peak lookup, and the rule that scales the DRAM traffic of one captured launch to the
timed launches only while the kernel's sources match the capture."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import rfdd_inputs as I  # noqa: E402


def test_workload_config_names_the_workload():
    w = I.workload("q1_3d_40")
    c = bench.workload_config(w, "mixed")
    assert c["name"] == "q1_3d_40" and c["n"] == 64000 and c["p"] == 8 and c["nev"] == 202
    assert c["n_nodes"] == 8 and c["precision"] == "mixed"
    assert "40x40x40" in c["workload"] and "model" not in c


def test_measured_peaks_has_the_denominators():
    peaks, src = bench.measured_peaks()
    assert src in ("measured", "fallback")
    for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained"):
        assert float(peaks[k]) > 0


def test_traffic_scaled_from_the_captured_ratio_only_for_the_captured_kernel(monkeypatch):
    monkeypatch.setattr(bench, "TC_TRAFFIC_RATIO", 1.25)
    monkeypatch.setattr(bench, "TC_TRAFFIC_SOURCES_SHA256", bench.kernel_sources_sha256())
    assert bench.tc_traffic_per_launch(1.0e9) == 1.25e9     # measured/model ratio x model bytes
    monkeypatch.setattr(bench, "TC_TRAFFIC_SOURCES_SHA256", "0" * 64)
    assert bench.tc_traffic_per_launch(1.0e9) is None       # the kernel changed since the capture
    monkeypatch.setattr(bench, "TC_TRAFFIC_RATIO", None)
    monkeypatch.setattr(bench, "TC_TRAFFIC_SOURCES_SHA256", bench.kernel_sources_sha256())
    assert bench.tc_traffic_per_launch(1.0e9) is None       # nothing captured


def test_kernel_hash_covers_the_kernel_sources():
    h = bench.kernel_sources_sha256()
    assert h == bench.kernel_sources_sha256() and len(h) == 64
    assert bench.kernel_sources_sha256(("tc_gemm.cu",)) != h


def test_reference_arm_other_ranks_exit_without_work():
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
