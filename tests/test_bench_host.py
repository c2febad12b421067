"""Host-side pieces of bench.py that need no GPU: the clock sampler's parsing
of nvidia-smi samples (median SM clock, maximum clock, throttle reasons) run
against a stand-in nvidia-smi on PATH, its behaviour when nvidia-smi is
missing, the GPU index under CUDA_VISIBLE_DEVICES, and the timed-region
status names."""
import os
import stat

import pytest

import bench

FAKE = """#!/bin/sh
echo "0, 2070, 2070, 812.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
echo "0, 2055, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
echo "0, 2070, 2070, 1388.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
echo "garbage line"
exec sleep 30
"""


def test_clock_sampler_parses_samples(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    cs = bench.ClockSampler(0)
    cs.start()
    out = cs.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    cs = bench.ClockSampler(0)
    cs.start()
    out = cs.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


@pytest.mark.parametrize("vis,rank,want", [("", 3, 3), ("4,5", 1, 5), ("2", 0, 2),
                                           ("GPU-abc", 1, 1)])
def test_gpu_index(monkeypatch, vis, rank, want):
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", vis)
    assert bench.gpu_index(rank) == want


def test_status_names():
    assert bench._status_names(0) == ["ok"]
    names = bench._status_names(1 | 2 | 4)
    assert len(names) == 3 and "ok" not in names


def test_updates_per_step_covers_min_time():
    import bench
    assert bench.updates_per_step(50, 120e-6, 1.2) == 200
    assert bench.updates_per_step(50, 1.0, 1.2) == 1
    assert bench.updates_per_step(3, 0.0, 0.1) >= 1


def test_iterations_run_from_merits():
    import bench
    assert bench.iterations_run([0.0] * 11, 10) == 0                 # safe V+
    assert bench.iterations_run([5.0, 2.0, 0.0] + [0.0] * 8, 10) == 2
    assert bench.iterations_run([5.0, 4.0, 4.0] + [4.0] * 8, 10) == 1  # line search stalled
    assert bench.iterations_run([float(10 - i) for i in range(11)], 10) == 10
