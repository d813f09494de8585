"""bench.py's clock record, on CPU: the sampler runs nvidia-smi during the
timed region and reports the median SM clock under load, the largest
maximum clock and every throttle reason seen active.  Here a stand-in
nvidia-smi on PATH prints a fixed CSV stream."""
import os
import stat

import bench

LINES = [
    "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 2055, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2070, 2070, 1390.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "garbage line",
    "0, [N/A], 2070, 1390.1, 0x0, Not Active, Not Active, Not Active, Not Active",
]


def fake_smi(tmp_path, lines):
    exe = tmp_path / "nvidia-smi"
    body = "\n".join(f"echo '{s}'" for s in lines)
    exe.write_text(f"#!/bin/sh\n{body}\nexec sleep 30\n")
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_median_max_and_reasons(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", fake_smi(tmp_path, LINES) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    r = s.stop()
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_thermal_slowdown_is_reported(tmp_path, monkeypatch):
    lines = ["0, 1500, 2070, 900.0, 0x40, Not Active, Active, Not Active, Not Active"]
    monkeypatch.setenv("PATH", fake_smi(tmp_path, lines) + os.pathsep + os.environ["PATH"])
    r = bench.ClockSampler(0).stop()
    assert r["sm_mhz"] == 1500.0 and r["reasons"] == ["hw_thermal_slowdown"]


def test_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    r = bench.ClockSampler(0).stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]
