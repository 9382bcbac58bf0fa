"""Host logic of bench.py that needs no GPU: clock-sample parsing, the roofline figures,
the peak lookup and capacity growth after an overflow (CPU only)."""
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


class _Sizes:
    Nv, E, F = 1000, 3000, 2000


def test_roofline_of_the_fp64_evaluation():
    """eval_barrier: achieved = pairs per launch x FP64 flops per pair / launch time, against
    the FP64 peak of 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz; traffic from the per-pair
    ncu figure."""
    r = bench.roofline_figure("eval_barrier", total_ms=20.0, launches=10, steps=10,
                              pairs_per_step=1e5, cand_per_step=1e6, sc=_Sizes)
    ach = 1e5 * bench.FP64_FLOPS_PER_PAIR / 2e-3 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - ach) <= 1e-12 * ach
    assert abs(r["peak"] - 152 * 4 * 2.07e9 / 1e12) <= 1e-12
    assert abs(r["frac"] - ach / r["peak"]) <= 1e-12
    assert r["traffic"] == bench.NCU_TRAFFIC_PER_UNIT["eval_barrier"] * 1e5
    # two launches per step split the step's pairs
    r2 = bench.roofline_figure("eval_barrier", total_ms=20.0, launches=20, steps=10,
                               pairs_per_step=1e5, cand_per_step=1e6, sc=_Sizes)
    assert abs(r2["achieved"] - ach) <= 1e-12 * ach


def test_roofline_of_a_memory_bound_kernel(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: (6000.0, "measured"))
    r = bench.roofline_figure("bvh_query", total_ms=5.0, launches=10, steps=10,
                              pairs_per_step=1e5, cand_per_step=1e6, sc=_Sizes)
    b = 0.5 * (32 * 1000 + 72 * 3000 + 64 * 5000 + 8 * 1e6)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6000.0
    assert abs(r["achieved"] - b / 5e-4 / 1e9) <= 1e-9 and abs(r["frac"] - r["achieved"] / 6000.0) <= 1e-15
    assert r["peak_source"] == "measured"


def test_roofline_without_launches_and_peak_fallback(monkeypatch, tmp_path):
    r = bench.roofline_figure("bvh_query", 0.0, 0, 10, 1.0, 1.0, _Sizes)
    assert r["frac"] is None and r["achieved"] is None
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))          # no peaks file there
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6655.6}')
    assert bench.measured_peaks() == (6655.6, "measured")


def test_capacities_grow_only_where_the_device_overflowed():
    caps = dict(pair=100, cand=1000, rec=5000, bsr=50)
    out = bench._grow(caps, [0, 2000, 0, 40])
    assert out["pair"] == 100 and out["rec"] == 5000
    assert out["cand"] == int(1.3 * 2000) + 1024
    assert out["bsr"] == max(50, int(1.3 * 40) + 1024)
    assert caps["cand"] == 1000                                 # the input is not modified


def test_cpu_leg_sample_with_every_query_is_the_whole_contact_set():
    """The CPU baseline's sampled stage, given every vertex and edge as a query, evaluates
    exactly the contact set (EE pairs with both sides queried counted once)."""
    import oracle
    from paper_2409_16385_gb300 import scenes
    sc = scenes.make_config(2, small=True)
    n, dt, n_cand = bench.oracle_sample(sc, 3, 1.0)
    full = oracle.pairs(sc, oracle.embed(sc, sc.iterate(3)))
    assert n == len(full["type"]) > 0 and dt > 0 and n_cand > 0
