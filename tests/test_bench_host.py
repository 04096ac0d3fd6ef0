"""Host-side pieces of bench.py that need no GPU: the clock record keeps the
nvidia-smi samples taken inside the timed region."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(sm, mx, power_cap="Not Active", thermal="Not Active", ts=""):
    return ["0", str(sm), str(mx), "900.0", "0x0", "Not Active", "Not Active", thermal, power_cap, ts]


def test_clock_samples_inside_the_timed_region_only():
    rows = [(10.0, _row(1200, 2070)), (11.0, _row(2070, 2070)), (11.2, _row(2055, 2070, power_cap="Active")),
            (11.4, _row(2070, 2070)), (13.0, _row(900, 2070, thermal="Active"))]
    ck = bench.ClockSampler.summarize(rows, 10.9, 11.5)
    assert ck["samples"] == 3 and ck["sm_mhz"] == 2070.0 and ck["sm_max_mhz"] == 2070.0
    assert ck["reasons"] == ["sw_power_cap"] and ck["window"] == "timed region"
    # no sample inside: every sample is summarised and the record says so
    ck = bench.ClockSampler.summarize(rows, 20.0, 21.0)
    assert ck["samples"] == 5 and "none inside" in ck["window"]
    assert ck["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]


def test_clock_sample_time_from_the_nvidia_smi_timestamp():
    t = datetime.datetime(2026, 12, 3, 11, 45, 1, 250000)
    got = bench.ClockSampler.sample_time(_row(2070, 2070, ts=t.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]), 0.0)
    assert abs(got - t.timestamp()) < 1e-6
    assert bench.ClockSampler.sample_time(_row(2070, 2070, ts="n/a"), 42.0) == 42.0  # else the arrival time
    assert bench.ClockSampler.sample_time(_row(2070, 2070)[:9], 7.0) == 7.0
