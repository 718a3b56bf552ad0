"""The bench's summary of the nvidia-smi clock samples taken during its timed
region: median SM clock, maximum clock, the throttle reasons that were
active (the ones that reject a run, and the power cap, which is noted).
No GPU: the samples are text."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_summary_of_samples():
    lines = [
        "2070, 2070, 812.4, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "1980, 2070, 1402.1, 0x0000000000000008, Active, Not Active, Not Active, Not Active\n",
        "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active\n",   # unreadable
        "short line\n",
    ]
    c = bench.ClockSampler.summarize(lines)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples():
    c = bench.ClockSampler.summarize([])
    assert c == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
