"""Host-side arithmetic of the benchmark (no GPU): the algorithmic bytes and FLOPs its
roofline figures divide by, the peaks it divides into, and the rule that a recorded DRAM
traffic or accuracy figure is reported only for the source it was taken on."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2504_10539_gb300 import workloads as wl  # noqa: E402


def test_bytes_per_update_follow_the_storage_layouts():
    # two-lattice push streaming: an update reads and writes each stored plane once
    assert bench.BYTES_PER_UPDATE[wl.F64] == 2 * 9 * 8
    assert bench.BYTES_PER_UPDATE[wl.F32] == 2 * 9 * 4
    assert bench.BYTES_PER_UPDATE[wl.F16_OFFSET] == 2 * 10 * 2   # nine offsets and the reference density


def test_training_flops_per_sample_follow_the_network():
    d = wl.MLP_DIMS
    fwd = sum(d[l] * d[l + 1] for l in range(len(d) - 1))
    back = sum(d[l] * d[l + 1] for l in range(1, len(d) - 1))   # nothing flows back into the 2 coordinates
    assert (fwd, back) == (33088, 32960)
    # value and two input tangents, each forward, backward to the inputs and weight gradient
    assert bench.TRAIN_FLOP_PER_SAMPLE == 2 * 3 * (fwd + back + fwd)


def test_peaks_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    assert bench.measured_peaks_bf16() == (1900.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6781.4, "bf16_tflops": 1912.7}))
    assert bench.measured_peaks() == (6781.4, "measured")
    assert bench.measured_peaks_bf16() == (1912.7, "measured")


def test_recorded_traffic_only_for_the_kernel_it_was_taken_on(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("f16_offset_batch", 100) is None           # no record
    (tmp_path / "profiles").mkdir()
    p = tmp_path / "profiles" / "step_kernel_traffic.json"
    rec = {"f16_offset_batch": {"dram_bytes_per_cell_update": 39.0, "kernel_sha1": bench.step_kernel_hash()}}
    p.write_text(json.dumps(rec))
    assert bench.profiled_traffic("f16_offset_batch", 1000) == 39000.0     # scaled by the cells updated
    assert bench.profiled_traffic("f32_field", 1000) is None                # no entry for that workload
    rec["f16_offset_batch"]["kernel_sha1"] = "0" * 16                       # taken on another source
    p.write_text(json.dumps(rec))
    assert bench.profiled_traffic("f16_offset_batch", 1000) is None


def test_accuracy_record_marked_stale_on_another_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.accuracy_record() is None
    (tmp_path / "profiles").mkdir()
    p = tmp_path / "profiles" / "accuracy_full_length.json"
    p.write_text(json.dumps({"source_sha1": bench.library_hash(), "C2": {}}))
    assert bench.accuracy_record()["stale"] is False
    p.write_text(json.dumps({"source_sha1": "0" * 16, "C2": {}}))
    assert bench.accuracy_record()["stale"] is True


def test_step_kernel_hash_covers_only_the_step_sources():
    from paper_2504_10539_gb300 import build as PB
    assert bench.step_kernel_hash() == PB.source_hash(("pl_step.cu", "pl_device.cuh", "pl_kernels.h"))
    assert bench.library_hash() == PB.source_hash() != bench.step_kernel_hash()


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on host cores and prints one JSON line with
    the benchmark's metric, its own CPU-baseline description and an end-to-end figure without
    device copies."""
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--lattices", "8"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "MLUPS" and d["unit"] == "MLUPS"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"] == "batch_8" and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
