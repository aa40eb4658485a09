"""The bench's clock sampler (host logic, no GPU): a stand-in for nvidia-smi
prints CSV lines at a fixed period, idle clocks before the timed region opens
and loaded clocks inside it; only the samples inside the region count."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

# prints "index, sm, max, power, active, hw, hw_thermal, sw_thermal, sw_power_cap"
# every 20 ms: 2070 MHz while the file `flag` exists, 345 MHz otherwise;
# sw_power_cap Active on every fifth loaded line
FAKE = r"""
import os, sys, time
flag = sys.argv[1]
k = 0
while True:
    loaded = os.path.exists(flag)
    cap = "Active" if (loaded and k % 5 == 4) else "Not Active"
    sm = 2070 if loaded else 345
    print("0, %d, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, %s" % (sm, cap), flush=True)
    k += loaded
    time.sleep(0.02)
"""


def _sampler(tmp_path, period_ms=20):
    script = tmp_path / "fake_smi.py"
    script.write_text(FAKE)
    flag = tmp_path / "loaded"
    return bench.ClockSampler(0, period_ms=period_ms, cmd=[sys.executable, str(script), str(flag)]), flag


def test_only_samples_inside_the_region_count(tmp_path):
    s, flag = _sampler(tmp_path)
    s.start()
    assert s.lines, "start() returns once the sampler has printed"
    time.sleep(0.2)                          # idle samples before the region
    flag.write_text("1")
    time.sleep(0.05)
    s.begin()
    time.sleep(0.5)
    clk = s.stop()
    assert clk["sm_mhz"] == 2070.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["samples"] >= 10
    assert clk["reasons"] == ["sw_power_cap"]


def test_short_region_takes_the_next_sample(tmp_path):
    s, flag = _sampler(tmp_path, period_ms=200)   # region much shorter than the nominal period
    flag.write_text("1")
    s.start()
    time.sleep(0.1)
    s.begin()
    clk = s.stop()
    assert clk is not None and clk["samples"] >= 1 and clk["sm_mhz"] == 2070.0


def test_parse_rejects_malformed_lines():
    assert bench.ClockSampler.parse("garbage") is None
    assert bench.ClockSampler.parse("0, [N/A], 2070, 1, 0, a, b, c, d") is None
    sm, mx, act = bench.ClockSampler.parse("0, 1980, 2070, 1, 0x4, Not Active, Active, Not Active, Active")
    assert (sm, mx) == (1980.0, 2070.0) and act == {"hw_thermal_slowdown", "sw_power_cap"}


def test_missing_sampler_gives_none():
    s = bench.ClockSampler(0, cmd=["/nonexistent/nvidia-smi-stand-in"])
    s.start()
    s.begin()
    assert s.stop() is None
