"""Host logic of bench.py that needs no GPU.  No GPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_clock_summary_from_nvidia_smi_lines():
    """bench.py's `clocks` field from nvidia-smi samples: the median under
    load (idle samples left out), the maximum clock, the slowdown reasons
    seen active (sw_power_cap kept as a note), malformed lines skipped."""
    sys.path.insert(0, ROOT)
    import bench

    n = "Not Active"
    lines = ["0, 2070, 2070, 900.1, 0x0, %s, %s, %s, %s\n" % (n, n, n, n),
             "0, 2055, 2070, 1100.0, 0x4, %s, %s, %s, Active\n" % (n, n, n),
             "0, 345, 2070, 120.0, 0x1, %s, %s, %s, %s\n" % (n, n, n, n),  # idle
             "0, 2070, 2070, 1200.0, 0x0, %s, %s, %s, %s\n" % (n, n, n, n),
             "garbage\n"]
    c = bench.parse_clock_lines(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}
    hot = ["0, 1500, 2070, 1300, 0x8, Active, %s, Active, %s\n" % (n, n)]
    assert bench.parse_clock_lines(hot)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.parse_clock_lines([]) is None
    assert bench.parse_clock_lines(["0, [N/A], [N/A], 1, 0x0, %s, %s, %s, %s\n" % (n, n, n, n)])["sm_mhz"] is None
