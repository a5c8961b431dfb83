"""bench.py's reading of the clock samples it takes during the timed steps.

A timed run whose samples show a hardware or thermal slowdown is rejected, so
the parser must report every throttle reason it sees, the median SM clock
under load and the maximum clock; rows that are not samples (a header, a
truncated line, "[N/A]" fields) are skipped.  No GPU is involved: the
samples are written by the test in nvidia-smi's CSV form.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def write(tmp_path, rows):
    p = tmp_path / "clocks.csv"
    p.write_text("".join(r + "\n" for r in rows))
    return str(p)


def row(sm, mx=2070, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return "0, %s, %s, 900.5, 0x0, %s, %s, %s, %s" % (sm, mx, hw, hwt, swt, cap)


def test_median_and_no_reason(tmp_path):
    c = bench.parse_clocks(write(tmp_path, [row(2070), row(2055), row(2070), row(1980)]))
    assert c == {"sm_mhz": 2062.5, "sm_max_mhz": 2070.0, "reasons": [], "samples": 4}


def test_every_reason_is_reported(tmp_path):
    rows = [row(2070), row(1800, hw="Active"), row(1700, hwt="Active"), row(1900, swt="Active"),
            row(2000, cap="Active")]
    c = bench.parse_clocks(write(tmp_path, rows))
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert c["samples"] == 5 and c["sm_mhz"] == 1900.0


def test_rows_that_are_not_samples_are_skipped(tmp_path):
    rows = ["index, clocks.current.sm [MHz], clocks.max.sm [MHz]", "0, 2070", row("[N/A]"), row(2070)]
    c = bench.parse_clocks(write(tmp_path, rows))
    assert c["samples"] == 1 and c["sm_mhz"] == 2070.0


def test_no_samples(tmp_path):
    assert bench.parse_clocks(write(tmp_path, [])) is None
