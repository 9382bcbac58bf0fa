"""Host logic of bench.py that needs no GPU: the clock-sample parsing (CPU only)."""
import datetime

import bench


def _line(t, sm, mx, hw="Not Active", thermal="Not Active", sw_thermal="Not Active", power="Not Active"):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{ts}, 0, {sm}, {mx}, 700.0, 0x0, {hw}, {thermal}, {sw_thermal}, {power}"


def test_median_and_reasons():
    text = "\n".join([_line(100.0, 2070, 2070), _line(100.1, 1980, 2070, power="Active"),
                      _line(100.2, 2070, 2070)])
    r = bench.parse_clock_samples(text)
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_window_keeps_only_the_timed_region():
    """Samples taken before the timed region (idle clocks) or after it do not count."""
    text = "\n".join([_line(99.0, 345, 2070), _line(100.02, 2070, 2070), _line(100.3, 2070, 2070),
                      _line(101.5, 345, 2070, hw="Active")])
    r = bench.parse_clock_samples(text, window=(100.0, 100.5))
    assert r["samples"] == 2 and r["sm_mhz"] == 2070.0 and r["reasons"] == []


def test_no_sample_in_the_window():
    text = _line(99.0, 2070, 2070)
    r = bench.parse_clock_samples(text, window=(100.0, 100.1))
    assert r["samples"] == 0 and r["sm_mhz"] is None and r["reasons"] == ["no samples"]


def test_malformed_lines_are_skipped():
    text = "garbage\n" + _line(100.0, "[N/A]", 2070) + "\n" + _line(100.05, 2000, 2070)
    r = bench.parse_clock_samples(text)
    assert r["samples"] == 1 and r["sm_mhz"] == 2000.0
