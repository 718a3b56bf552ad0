"""Host-side parts of bench.py, no GPU: the summary of the nvidia-smi clock
samples taken during the timed region (median SM clock, maximum clock, the
throttle reasons that were active), given as text; and the reference arm,
which times the FP64 oracle on the host and prints the contract's JSON line."""
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


def test_reference_arm_prints_its_json_line():
    """bench.py --impl reference times the FP64 oracle on a crop of the workload
    on the host and prints one JSON line with the contract's keys."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "MP/s"
    assert line["higher_is_better"] is True and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]
