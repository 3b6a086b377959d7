"""bench.py's clock record on the host: parsing of the nvidia-smi samples taken during the timed
region (median SM clock, maximum, throttle reasons), and the sampler's stop path with a stand-in
process in place of nvidia-smi."""
import os
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

ROWS = """0, 2070, 2070, 812.4, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
0, 1980, 2070, 1391.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, 2070, 2070, 905.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
0, [N/A], 2070, 0.0, [N/A], [N/A], [N/A], [N/A], [N/A]
0, 2070, 2070
"""


def test_summary_of_samples():
    c = bench.summarise_clocks(ROWS)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_throttle_reasons_are_named():
    line = "0, 1500, 2070, 700.0, 0x48, Active, Active, Not Active, Not Active"
    c = bench.summarise_clocks(line)
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and c["sm_mhz"] == 1500.0


def test_no_parsable_sample_gives_none():
    assert bench.summarise_clocks("") is None
    assert bench.summarise_clocks("0, [N/A], [N/A], 0, 0, a, b, c, d") is None


def test_stop_reads_and_removes_the_sample_file():
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    s.f = open(s.path, "w")
    s.f.write(ROWS)
    s.f.flush()
    s.proc = subprocess.Popen([sys.executable, "-c", "import time; time.sleep(30)"])
    c = s.stop()
    assert c["samples"] == 3 and c["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(s.path)
    assert s.proc.poll() is not None
