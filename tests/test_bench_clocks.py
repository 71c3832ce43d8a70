"""bench.py's summary of the nvidia-smi clock samples taken during the timed
region (CPU only, synthetic sample rows)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(sm, smax, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return f"{sm}, {smax}, 950.00, 0x0000000000000000, " + ", ".join(flags) + "\n"


def test_median_under_load_and_no_reasons():
    lines = [_row(345, 2070)] + [_row(2070, 2070)] * 5 + [_row(2055, 2070)] * 2
    out = bench.summarize_clocks(lines)
    assert out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2070.0           # the idle sample below half the maximum is left out
    assert out["samples"] == 8 and out["reasons"] == []


def test_reasons_seen_active_are_reported():
    lines = [_row(2070, 2070), _row(1980, 2070, ("sw_power_cap",)),
             _row(1500, 2070, ("hw_slowdown", "sw_power_cap"))]
    out = bench.summarize_clocks(lines)
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == 1980.0


def test_unparsable_rows_are_skipped():
    lines = ["[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]\n", "garbage\n", "\n",
             _row(2070, 2070)]
    out = bench.summarize_clocks(lines)
    assert out["samples"] == 1 and out["sm_mhz"] == 2070.0
    empty = bench.summarize_clocks([])
    assert empty["sm_mhz"] is None and empty["samples"] == 0
