"""bench.py's clock record: only nvidia-smi samples taken inside the timed
region count, by nvidia-smi's own timestamps.  Runs on the CPU with a fake
nvidia-smi that prints samples the way the real one does."""
import datetime
import os
import stat
import sys
import time

import bench


def _line(t, sm=2070, mx=2070, reasons=("Not Active",) * 4):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return "%s, 0, %d, %d, 500.00, 0x0000000000000000, %s" % (ts, sm, mx, ", ".join(reasons))


def test_summary_keeps_the_samples_inside_the_region():
    t = 1_800_000_000.0
    lines = [_line(t - 1.0, sm=900, reasons=("Active", "Not Active", "Not Active", "Not Active")),
             _line(t + 0.10, sm=2070), _line(t + 0.15, sm=2055),
             _line(t + 0.20, sm=2070, reasons=("Not Active", "Not Active", "Not Active", "Active")),
             _line(t + 2.0, sm=1000, reasons=("Not Active", "Active", "Not Active", "Not Active")),
             "garbage", ""]
    s = bench.clock_summary(lines, t + 0.08, t + 0.21, slack=0.0)
    assert s["samples"] == 3 and s["samples_outside"] == 2
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]  # the hw_slowdown before and the thermal one after do not count
    # the slack widens the region by the sampling period on both sides
    assert bench.clock_summary(lines, t + 0.12, t + 0.13, slack=0.05)["samples"] == 2
    # no region: every sample counts
    allr = bench.clock_summary(lines)
    assert allr["samples"] == 5 and set(allr["reasons"]) == {"hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"}
    empty = bench.clock_summary(lines, t + 5.0, t + 6.0, slack=0.0)
    assert empty["samples"] == 0 and empty["sm_mhz"] is None


FAKE_SMI = r'''#!%s
import datetime, sys, time
period = int(sys.argv[sys.argv.index("-lms") + 1]) / 1000.0
assert "--query-gpu=" + %r in sys.argv
while True:
    ts = datetime.datetime.now().strftime("%%Y/%%m/%%d %%H:%%M:%%S.%%f")[:-3]
    print("%%s, 0, 2070, 2070, 612.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active" %% ts,
          flush=True)
    time.sleep(period)
'''


def test_sampler_records_the_region(tmp_path):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE_SMI % (sys.executable, bench.ClockSampler.Q))
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    c = bench.ClockSampler(0, exe=str(exe)).start()
    try:
        time.sleep(0.5)  # the warm-up
        c.begin()
        time.sleep(0.4)  # the timed region
        c.end()
    finally:
        c.stop()
    s = c.summary()
    assert s["samples"] >= 4, s  # one every 50 ms
    assert s["samples_outside"] >= 2, s  # the warm-up's samples are left out
    assert s["sm_mhz"] == 2070 and s["reasons"] == []


def test_sampler_without_nvidia_smi(tmp_path):
    c = bench.ClockSampler(0, exe=str(tmp_path / "missing")).start()
    c.begin()
    c.end()
    c.stop()
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "samples_outside": 0}
