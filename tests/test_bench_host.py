"""Host logic of bench.py (no GPU): the DRAM-traffic record is used only for
the scan source it was measured on, and the clock sampler's parsing of
nvidia-smi's CSV (against a fake nvidia-smi on PATH)."""
import hashlib
import json
import os
import stat
import time

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCAN = os.path.join(ROOT, "paper_2511_14955_gb300", "csrc", "ig_scan.cu")


def test_traffic_record_only_for_the_measured_source(tmp_path):
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    cur = hashlib.sha256(open(SCAN, "rb").read()).hexdigest()
    got = bench.traffic_record(SCAN)
    if rec["scan_kernel_sha256"] == cur:
        assert got == rec["dram_bytes_per_launch"] and got > 0
    else:
        assert got is None
    changed = tmp_path / "ig_scan.cu"
    changed.write_bytes(open(SCAN, "rb").read() + b"\n// changed\n")
    assert bench.traffic_record(str(changed)) is None
    assert bench.traffic_record(str(tmp_path / "missing.cu")) is None


def test_clock_sampler_parses_fake_nvidia_smi(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 1995, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "echo '0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo 'garbage line'\n"
                    "exec sleep 30\n")
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")
    cs = bench.ClockSampler(0)
    cs.start()
    time.sleep(0.5)
    out = cs.stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_passes_of():
    assert bench.passes_of(dict(n=8, base_n=3)) == 6
    assert bench.passes_of(dict(n=2, base_n=3)) == 1
