"""bench.py's clock sampler against a stand-in nvidia-smi on PATH (no GPU):
the median SM clock under load, the maximum clock and power, and the active
throttle reasons decoded from the bit mask."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

FAKE = """#!/bin/sh
# index, clocks.sm, clocks.max.sm, power.draw, clocks_event_reasons.active, utilization.gpu
echo "0, 1200, 2070, 150.0, 0x0000000000000001, 0"
while true; do
  echo "0, 2070, 2070, 900.5, 0x0000000000000004, 99"
  echo "0, 2055, 2070, 910.0, 0x0000000000000000, 97"
  sleep 0.05
done
"""


def test_clock_sampler_parses_samples(tmp_path, monkeypatch):
    import bench
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = bench.ClockSampler(0)
    c.start()
    time.sleep(0.5)
    out = c.stop()
    assert out is not None and out["samples"] >= 3
    assert out["samples_under_load"] == out["samples"] - 1   # the idle first line
    assert out["sm_max_mhz"] == 2070.0 and out["power_w_max"] == 910.0
    assert 2055.0 <= out["sm_mhz"] <= 2070.0
    assert out["reasons"] == ["sw_power_cap"]                 # gpu_idle is not a reason
    assert not os.path.exists(c.path)


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop() is None
    assert not os.path.exists(c.path)
