"""The benchmark's clock sampler (CPU only): a stand-in `nvidia-smi` on PATH
prints one CSV sample every 50 ms; the sampler must wait for the first one,
keep only the samples of the timed window and read the throttle reasons."""
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LINE = "0, 1980 MHz, 2070 MHz, 301.50 W, 0x4, Not Active, Not Active, Not Active, Active"


@pytest.fixture
def fake_smi(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(f"#!/bin/sh\nwhile true; do echo '{LINE}'; sleep 0.05; done\n")
    exe.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")
    return exe


def test_samples_of_the_timed_window(fake_smi):
    import bench

    c = bench.ClockSampler(0)
    c.start()
    assert c.lines, "start() returns once the first sample is in"
    w0 = time.time()
    time.sleep(0.4)
    w1 = time.time()
    time.sleep(0.3)  # samples after the window (beyond the grace) are dropped
    r = c.stop((w0, w1))
    assert r["window"] == "timed region"
    assert 4 <= r["samples"] <= 12
    assert r["sm_mhz"] == 1980.0 and r["sm_max_mhz"] == 2070.0 and r["power_w_max"] == 301.5
    assert r["reasons"] == ["sw_power_cap"]


def test_no_sample_in_the_window_falls_back_to_the_whole_run(fake_smi):
    import bench

    c = bench.ClockSampler(0)
    c.start()
    time.sleep(0.2)
    r = c.stop((0.0, 1.0))  # a window long past
    assert r["window"].startswith("whole run") and r["samples"] >= 2


def test_disabled_sampler_reports_nothing():
    import bench

    c = bench.ClockSampler(0, enabled=False)
    c.start()
    assert c.stop((0.0, 1.0)) is None
