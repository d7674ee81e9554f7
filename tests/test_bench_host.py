"""CPU checks of bench.py's host logic: the clock sampler's reading of
nvidia-smi rows (median and peak SM clock, which throttle reasons were
active)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self):
        pass


def _sample(rows):
    c = bench.ClockSampler(0)
    c.p = _Proc()
    c.f.write("".join(r + "\n" for r in rows))
    c.f.flush()
    return c.stop()


def test_clock_rows_give_median_peak_and_reasons():
    rows = ["0, 2032, 2032, 910.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2032, 1101.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2010, 2032, 1050.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"]
    out = _sample(rows)
    assert out["sm_mhz"] == 2010.0 and out["sm_max_mhz"] == 2032.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_thermal_and_hw_slowdown_are_reported():
    rows = ["0, 1500, 2032, 700.0, 0x0000000000000048, Active, Not Active, Active, Not Active",
            "0, 2032, 2032, 700.0, 0x0000000000000000, Not Active, Active, Not Active, Not Active"]
    out = _sample(rows)
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_unparseable_rows_are_skipped():
    rows = ["0, [N/A], 2032, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2000, 2032, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    out = _sample(rows)
    assert out["sm_mhz"] == 2000.0 and out["samples"] == 1 and out["reasons"] == []
