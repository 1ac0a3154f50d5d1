"""bench.py reports ncu-derived figures (DRAM traffic per launch, per-cell
arithmetic) only while they were taken on the current kernel sources: the
committed records carry a hash of those sources, and a record whose hash
differs reads as null.  CPU only."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_records_are_reported_only_for_their_sources(monkeypatch):
    """Every record carries the hash of the sources it was taken on; bench
    reports it exactly when that hash is the current one."""
    import json
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        traffic = json.load(f)
    for key, e in traffic.items():
        if not isinstance(e, dict):
            continue
        h = e["kernel_hash"]
        assert len(h) == 16 and int(h, 16) >= 0, key
        sources = bench.STEP3_SOURCES if key.startswith("d3q19") else bench.STEP_SOURCES
        monkeypatch.setattr(bench, "_kernel_hash", lambda s=bench.STEP_SOURCES, h=h: h)
        assert bench._traffic(key, sources) == e["dram_bytes_per_launch"], key
    with open(os.path.join(ROOT, "profiles", "ncu_alu.json")) as f:
        alu = json.load(f)
    monkeypatch.setattr(bench, "_kernel_hash", lambda s=bench.STEP_SOURCES: alu["kernel_hash"])
    a = bench._alu("f64")
    assert a is not None and a["fp64_ops"] > 0


def test_records_read_as_null_when_sources_change(monkeypatch):
    monkeypatch.setattr(bench, "_kernel_hash", lambda sources=bench.STEP_SOURCES: "0" * 16)
    assert bench._traffic("f32") is None
    assert bench._traffic("d3q19_f32", bench.STEP3_SOURCES) is None
    assert bench._alu("f32") is None


def test_hash_covers_every_step_source():
    csrc = os.path.join(ROOT, "paper_1507_03521_gb300", "csrc")
    for name in bench.STEP_SOURCES + bench.STEP3_SOURCES:
        assert os.path.exists(os.path.join(csrc, name)), name
    assert bench._kernel_hash() != bench._kernel_hash(bench.STEP3_SOURCES)


@pytest.mark.parametrize("key", ["f32", "f16s", "bf16s", "f64", "lag_f32", "slab_f32", "batch_f32"])
def test_traffic_records_are_near_the_algorithmic_bytes(key):
    import json
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        e = json.load(f)[key]
    assert 0.9 <= e["dram_bytes_per_launch"] / e["algorithmic"] <= 1.3, key


def test_clock_sampler_counts_samples_inside_the_region(tmp_path, monkeypatch):
    """The clock sampler with a stand-in nvidia-smi (one sample every
    10 ms): entering waits until sampling is live, and the samples stamped
    inside the timed region are counted with their throttle reasons."""
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\nwhile true; do\n"
                    "  echo '0, 1980, 2070, 950.5, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "  sleep 0.01\ndone\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    with bench.Clocks(0, interval_ms=10) as ck:
        time.sleep(0.2)
    s = ck.summary()
    assert s["samples"] >= 5, s
    assert s["sm_mhz"] == 1980.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
