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


PER_STEP = dict(pairs=1e5, ccd=2e4, cand_contact=1e6, cand_ccd=3e5)


def test_roofline_of_the_fp64_evaluation():
    """eval_barrier: achieved = pairs per launch x FP64 flops per pair / launch time, against
    the FP64 peak of 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz; traffic from the per-pair
    ncu figure; the live probe's rate is reported beside it."""
    r = bench.roofline_figure("eval_barrier", 20.0, 10, 10, PER_STEP, _Sizes, dict(tflops=1.2))
    ach = 1e5 * bench.FP64_FLOPS_PER_PAIR / 2e-3 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - ach) <= 1e-12 * ach
    assert abs(r["peak"] - 152 * 4 * 2.07e9 / 1e12) <= 1e-12
    assert abs(r["frac"] - ach / r["peak"]) <= 1e-12
    assert abs(r["frac_of_probe"] - ach / 1.2) <= 1e-12 and r["peak_probe"] == 1.2
    assert r["traffic"] == bench.NCU_TRAFFIC_PER_UNIT["eval_barrier"] * 1e5
    # two launches per step split the step's pairs
    r2 = bench.roofline_figure("eval_barrier", 20.0, 20, 10, PER_STEP, _Sizes)
    assert abs(r2["achieved"] - ach) <= 1e-12 * ach and "peak_probe" not in r2


def test_roofline_of_the_traversal_uses_both_traversals_candidates(monkeypatch):
    """bvh_query runs twice per step (contact set, CCD): its bytes per launch average the
    two launches' minimum traffic, each with its own candidate count."""
    monkeypatch.setattr(bench, "measured_peaks", lambda: (6000.0, "measured"))
    r = bench.roofline_figure("bvh_query", 5.0, 20, 10, PER_STEP, _Sizes)
    base = 32 * 1000 + 8 * 3000 + 64 * (2 * 2000 + 2 * 3000)
    b = 0.5 * ((base + 8 * 1e6) + (base + 8 * 3e5))
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6000.0
    assert abs(r["bytes_per_launch"] - b) <= 1e-9 * b
    assert abs(r["achieved"] - b / 2.5e-4 / 1e9) <= 1e-9 and abs(r["frac"] - r["achieved"] / 6000.0) <= 1e-15
    assert r["peak_source"] == "measured" and "latency-bound" in r["note"]


def test_roofline_without_launches_and_peak_fallback(monkeypatch, tmp_path):
    r = bench.roofline_figure("bvh_query", 0.0, 0, 10, PER_STEP, _Sizes)
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


def test_swept_overlap_matches_a_direct_box_test():
    """The host-side copy of the CCD's exact FP64 swept-box test, against boxes built
    pair by pair."""
    import numpy as np
    import oracle
    from paper_2409_16385_gb300 import scenes
    sc = scenes.make_config(1)
    x = oracle.embed(sc, sc.iterate(0))
    dx = oracle.embed(sc, sc.dq(0), displacement=True)
    rng = np.random.default_rng(1)
    n = 3000
    ct = rng.integers(0, 2, n).astype(np.int32)
    ci = np.where(ct == 0, rng.integers(0, sc.Nv, n), rng.integers(0, sc.E, n)).astype(np.int32)
    cj = np.where(ct == 0, rng.integers(0, sc.F, n), rng.integers(0, sc.E, n)).astype(np.int32)
    # random pairs (mostly far apart) and the contact pairs (close: mostly overlapping)
    near = oracle.pairs(sc, x)
    ct = np.concatenate([ct, near["type"]]).astype(np.int32)
    ci = np.concatenate([ci, near["i"]]).astype(np.int32)
    cj = np.concatenate([cj, near["j"]]).astype(np.int32)
    n = len(ct)
    cand = dict(type=ct, i=ci, j=cj)
    got = bench.swept_overlap(sc, x, dx, cand)
    for k in range(n):
        if ct[k] == 0:
            A, B = [ci[k]], list(sc.tris[cj[k]])
        else:
            A, B = list(sc.edges[ci[k]]), list(sc.edges[cj[k]])
        pa = np.concatenate([x[A], x[A] + dx[A]]); pb = np.concatenate([x[B], x[B] + dx[B]])
        ov = np.all(pa.min(0) <= pb.max(0)) and np.all(pb.min(0) <= pa.max(0))
        assert got[k] == ov, k
    assert 0 < got.sum() < n


def test_pair_split_counts_pairs_between_bodies():
    import numpy as np
    from paper_2409_16385_gb300 import scenes
    sc = scenes.make_config(1)                                  # sphere (body 0) on the pad (body 1)
    body = np.asarray(sc.body)
    v_sphere = int(np.nonzero(body == 0)[0][0])
    f_pad = int(np.nonzero(body[sc.tris[:, 0]] == 1)[0][0])
    f_sphere = int(np.nonzero(body[sc.tris[:, 0]] == 0)[0][-1])
    e_pad = int(np.nonzero(body[sc.edges[:, 0]] == 1)[0][0])
    e_sph = int(np.nonzero(body[sc.edges[:, 0]] == 0)[0][0])
    h = dict(type=np.array([0, 0, 1, 1]), i=np.array([v_sphere, v_sphere, e_sph, e_sph]),
             j=np.array([f_pad, f_sphere, e_pad, e_sph + 1]))
    assert bench.pair_split(sc, h) == dict(inter_body=2, intra_body=2)


def test_cpu_stage_baseline_runs_each_stage_on_the_given_lists():
    """The CPU legs time the oracle's evaluation and CCD stages over given lists (here the
    oracle's own, standing in for the GPU's), on all cores and on one core, and restore the
    thread count."""
    import oracle
    from paper_2409_16385_gb300 import scenes
    sc = scenes.make_config(2, small=True)
    x, xn = oracle.embed(sc, sc.iterate(3)), oracle.embed(sc, sc.iterate(sc.lag_of(3)))
    dx = oracle.embed(sc, sc.dq(3), displacement=True)
    prs, pn = oracle.pairs(sc, x), oracle.pairs(sc, xn)
    cand = dict(type=prs["type"], i=prs["i"], j=prs["j"])
    n0 = oracle.num_threads()
    r = bench.cpu_stage_baseline(sc, x, xn, dx, prs, pn, cand, budget_s=0.2)
    assert oracle.num_threads() == n0
    assert set(r) == {"eval_all", "eval_1core", "ccd_all", "ccd_1core"}
    assert r["eval_1core"]["threads"] == 1 and r["eval_all"]["threads"] == n0
    assert all(v["value"] > 0 for v in r.values())
    assert r["eval_all"]["list_pairs"] == len(prs["type"])
    e = bench.cpu_enumeration(sc, x, n_queries=50)
    assert e["pairs_found"] >= 0 and e["full_enumeration_s_estimate"] > 0


def test_classify_pairs_on_hand_built_configurations():
    """The bench's closest-feature classes on configurations whose answer is known."""
    import numpy as np

    class Sc:
        pass
    sc = Sc()
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0],              # triangle 0
                  [0.2, 0.2, 0.1],                              # 3: above the face
                  [0.5, -0.3, 0.1],                             # 4: beyond edge (0,1)
                  [-0.3, -0.3, 0.1],                            # 5: beyond vertex 0
                  [0.5, 0.5, 1.0], [0.5, 0.5, 2.0],             # 6-7: unused
                  [0.5, -1, 0.2], [0.5, 1, 0.2],                # 8-9: edge crossing over edge (0,1)
                  [0.5, 0.2, 0.3], [0.5, 2.0, 0.3],             # 10-11: T: endpoint 10 above edge (0,1) interior
                  [-1, 3, 0], [-1, 4, 0]], float)               # 12-13: edge beyond vertex 2 of edge (1,2)
    sc.tris = np.array([[0, 1, 2]])
    sc.edges = np.array([[0, 1], [8, 9], [10, 11], [12, 13], [1, 2]])
    sc.cage_idx = np.tile(np.arange(4), (len(x), 1))
    sc.cage_idx[12:] = -1
    h = dict(type=np.array([0, 0, 0, 1, 1, 1]), i=np.array([3, 4, 5, 0, 0, 4]), j=np.array([0, 0, 0, 1, 2, 3]))
    cls, nodes = bench.classify_pairs(sc, x, h)
    names = [bench.PAIR_CLASSES[c] for c in cls]
    assert names == ["pt_face", "pt_edge", "pt_vertex", "ee_interior", "ee_edge", "ee_vertex"], names
    assert list(nodes) == [4, 4, 4, 4, 4, 4]


def test_roofline_of_the_overlapped_evaluation():
    """eval_kernels: the barrier kernel's FP64 flops (friction of the pairs that carry it
    included) and DRAM bytes per contact pair, over the span of the overlapped launches."""
    ps = dict(PER_STEP, friction_items=0.5e5)
    r = bench.roofline_figure("eval_kernels", 20.0, 10, 10, ps, _Sizes)
    ach = 1e5 * bench.FP64_FLOPS_PER_PAIR / 2e-3 / 1e12
    assert abs(r["achieved"] - ach) <= 1e-12 * ach and r["bound"] == "alu"
    tr = bench.NCU_TRAFFIC_PER_UNIT["eval_barrier"] * 1e5
    assert abs(r["traffic"] - tr) <= 1e-9 * tr
