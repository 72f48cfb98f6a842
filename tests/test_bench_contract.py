"""bench.py on the CPU: the reference arm's JSON line (the oracle timed on
host cores) carries every key of the contract, and the dominant kernel's
DRAM traffic is reported only while the kernel sources match the capture."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith(bench.WORKLOAD)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_traffic_follows_the_kernel_source_hash(tmp_path, monkeypatch):
    rec = {"kernel": "res_sweep_kernel", "source_hash": bench.kernel_source_hash(), "dram_bytes_per_launch": 12345}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_record("res_sweep_kernel")["dram_bytes_per_launch"] == 12345
    assert bench.measured_record("strip_sweep_kernel") is None  # another kernel
    rec["source_hash"] = "0" * 16  # sources changed since the capture
    f.write_text(json.dumps(rec))
    assert bench.measured_record("res_sweep_kernel") is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.measured_record("res_sweep_kernel") is None


def test_kernel_source_hash_is_stable_and_covers_the_resident_sources():
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    csrc = os.path.join(ROOT, "paper_2009_12638_gb300", "csrc")
    for name in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(csrc, name)), name
    assert "ms_resident.cuh" in bench.KERNEL_SOURCES and "ms_resident_kernels.cuh" in bench.KERNEL_SOURCES
