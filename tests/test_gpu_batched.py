"""Batched scenes: many independent grasp scenes concatenated into one scene with one group
per scene, evaluated by one set of launches (and by one CUDA graph replay), compared scene
by scene with the plain path run on each scene alone.

The comparison is bitwise: a scene's positions are the same numbers in both runs (the
batch stores each scene already translated to its grid slot), the contact set is exact,
every reduction sums a segment's records in the order of its own pairs, and the per-group
energy uses the same fixed-order warp sum on both sides.  The plain path is itself held to
the oracle in the parity tests; two scenes of the batch are checked against the oracle here
as well.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_2409_16385_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@functools.lru_cache(maxsize=None)
def _batch():
    return scenes.make_config(4, small=True)


def _contact_scene(sc, groups=None):
    from paper_2409_16385_gb300 import ContactScene
    rec = (1 << 24) if groups is not None else (1 << 21)
    cs = ContactScene(sc, pair_capacity=1 << 20, bsr_capacity=1 << 21, rec_capacity=rec)
    if groups is not None:
        cs.set_groups(*groups)
    return cs


def _step(cs, sc, t, outs=None):
    """One contact stage at iterate t: lag at the lagged iterate, pairs, evaluation,
    per-group energy, CCD along dq(t), per-group alpha."""
    q = _t(sc.iterate(t))
    qn = _t(sc.iterate(sc.lag_of(t)))
    dq = _t(sc.dq(t))
    lag = cs.friction_lag(qn, cs.build_candidates(qn, out=cs.new_pairs()))
    pairs = cs.build_candidates(q)
    E, g, H = cs.eval_contact(q, pairs, lag)
    Eg = cs.group_energy()
    x = cs.embed(q)
    dx = cs.embed(dq, displacement=True)
    alpha = cs.accd_toi(x, dx)
    ag = cs.group_alpha()
    torch.cuda.synchronize()
    st = cs.status()
    assert st["flags"] == 0, st
    return dict(pairs=pairs.host(), lag=lag.host(), E=E.item(), g=g.cpu().numpy(), H=H.host(), Eg=Eg.cpu().numpy(),
                alpha=alpha.item(), ag=ag.cpu().numpy())


def _part_pairs(P, b, s):
    """Scene s's pairs out of the batch's list, renumbered to the scene's own ids."""
    v0, nv = b.vertex_ranges[s]
    f0, nf = b.tri_ranges[s]
    e0, ne = b.edge_ranges[s]
    ty, i, j, d = P["type"], P["i"], P["j"], P["d"]
    pt = (ty == 0) & (i >= v0) & (i < v0 + nv)
    ee = (ty == 1) & (i >= e0) & (i < e0 + ne)
    # the group filter keeps both ends of every pair in one scene
    assert np.all((j[pt] >= f0) & (j[pt] < f0 + nf))
    assert np.all((j[ee] >= e0) & (j[ee] < e0 + ne))
    sel = pt | ee
    ii = np.where(ty[sel] == 0, i[sel] - v0, i[sel] - e0)
    jj = np.where(ty[sel] == 0, j[sel] - f0, j[sel] - e0)
    return ty[sel], ii.astype(np.int32), jj.astype(np.int32), d[sel]


def _part_bsr(H, b, s):
    n0, ns = b.node_ranges[s]
    rp, col, val = H["row_ptr"], H["col"], H["val"]
    lo, hi = rp[n0], rp[n0 + ns]
    c = col[lo:hi]
    assert np.all((c >= n0) & (c < n0 + ns)), "a Hessian block joins two scenes"
    return (rp[n0:n0 + ns + 1] - lo).astype(np.int32), (c - n0).astype(np.int32), val[lo:hi]


@pytest.mark.parametrize("t", [4, 17])
def test_batch_matches_plain_path_scene_by_scene(t):
    b = _batch()
    cs = _contact_scene(b, (b.body, b.n_scenes))
    rb = _step(cs, b, t)
    npairs = 0
    for s in range(b.n_scenes):
        one = b.part_scene(s)
        r1 = _step(_contact_scene(one), one, t)
        ty, i, j, d = _part_pairs(rb["pairs"], b, s)
        p1 = r1["pairs"]
        assert np.array_equal(ty, p1["type"]) and np.array_equal(i, p1["i"]) and np.array_equal(j, p1["j"]), s
        assert np.array_equal(d, p1["d"]), s
        npairs += len(ty)
        n0, ns = b.node_ranges[s]
        assert np.array_equal(rb["g"][n0:n0 + ns], r1["g"]), s
        rp, col, val = _part_bsr(rb["H"], b, s)
        assert np.array_equal(rp, r1["H"]["row_ptr"]) and np.array_equal(col, r1["H"]["col"]), s
        assert np.array_equal(val, r1["H"]["val"]), s
        assert rb["Eg"][s] == r1["Eg"][0], (s, rb["Eg"][s], r1["Eg"][0])
        assert abs(r1["Eg"][0] - r1["E"]) <= 1e-12 * abs(r1["E"]) + 1e-300
        assert rb["ag"][s] == r1["alpha"], (s, rb["ag"][s], r1["alpha"])
    assert npairs == len(rb["pairs"]["type"]), "pairs outside every scene"
    assert rb["alpha"] == rb["ag"].min()
    assert abs(rb["Eg"].sum() - rb["E"]) <= 1e-12 * abs(rb["E"])
    assert npairs > 100 * b.n_scenes // 4


@pytest.mark.parametrize("s", [0, 5])
def test_batch_scene_against_oracle(s):
    """Two scenes of the batch, evaluated in the batch, against the oracle on that scene."""
    b = _batch()
    t = 9
    cs = _contact_scene(b, (b.body, b.n_scenes))
    rb = _step(cs, b, t)
    one = b.part_scene(s)
    p = one.params
    x = oracle.embed(one, one.iterate(t))
    xn = oracle.embed(one, one.iterate(one.lag_of(t)))
    po, pon = oracle.pairs(one, x), oracle.pairs(one, xn)
    ro = oracle.eval_contact(one, x, po, oracle.friction_lag(one, xn, pon))
    ty, i, j, d = _part_pairs(rb["pairs"], b, s)
    kg = set(zip(ty.tolist(), i.tolist(), j.tolist()))
    ko = set(zip(po["type"].tolist(), po["i"].tolist(), po["j"].tolist()))
    dd = dict(zip(zip(po["type"].tolist(), po["i"].tolist(), po["j"].tolist()), po["d"].tolist()))
    dg = dict(zip(zip(ty.tolist(), i.tolist(), j.tolist()), d.tolist()))
    for k in kg ^ ko:
        dk = dg.get(k, dd.get(k))
        assert abs(dk - p["dhat"]) <= 1e-12 * p["dhat"], k
    n0, ns = b.node_ranges[s]
    g = rb["g"][n0:n0 + ns]
    assert np.abs(g - ro["g"]).max() <= 1e-9 * np.abs(ro["g"]).max()
    assert abs(rb["Eg"][s] - ro["E"]) <= 1e-9 * abs(ro["E"])
    rp, col, val = _part_bsr(rb["H"], b, s)
    hg = {(r, int(col[k])): val[k] for r in range(ns) for k in range(rp[r], rp[r + 1])}
    ho = {(int(a), int(c)): v for a, c, v in zip(ro["I"], ro["J"], ro["V"])}
    assert set(hg) == set(ho)
    hs = max(np.abs(v).max() for v in ho.values())
    assert max(np.abs(hg[k] - ho[k]).max() for k in ho) <= 1e-9 * hs
    ao = oracle.accd(one, x, oracle.embed(one, one.dq(t), displacement=True))["alpha"]
    assert rb["ag"][s] <= ao and ao - rb["ag"][s] <= 1e-6


def test_graph_replay_matches_eager():
    """The whole batched stage captured once in a CUDA graph and replayed on new inputs
    gives bitwise the eager results."""
    b = _batch()
    cs = _contact_scene(b, (b.body, b.n_scenes))
    cs.set_rebuild_interval(1)
    t0, t1 = 4, 17
    q = _t(b.iterate(t0)); qn = _t(b.iterate(b.lag_of(t0))); dq = _t(b.dq(t0))
    pn, pr, lag, H = cs.new_pairs(), cs.new_pairs(), cs.new_lag(), cs.new_bsr()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros((b.Ns, 3), dtype=torch.float64, device="cuda")
    Eg = torch.zeros(b.n_scenes, dtype=torch.float64, device="cuda")
    ag = torch.zeros(b.n_scenes, dtype=torch.float64, device="cuda")
    x = torch.zeros((b.Nv, 3), dtype=torch.float64, device="cuda")
    dx = torch.zeros_like(x)
    alpha = torch.zeros(1, dtype=torch.float64, device="cuda")

    def stage():
        cs.build_candidates(qn, out=pn)
        cs.friction_lag(qn, pn, out=lag)
        cs.build_candidates(q, out=pr)
        cs.eval_contact(q, pr, lag, E=E, g_r=g, H=H)
        cs.group_energy(out=Eg)
        cs.embed(q, out=x)
        cs.embed(dq, out=dx, displacement=True)
        cs.accd_toi(x, dx, alpha=alpha)
        cs.group_alpha(out=ag)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        stage()                                  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        stage()
    q.copy_(_t(b.iterate(t1))); qn.copy_(_t(b.iterate(b.lag_of(t1)))); dq.copy_(_t(b.dq(t1)))
    graph.replay()
    torch.cuda.synchronize()
    got = (E.cpu().numpy().tobytes(), g.cpu().numpy().tobytes(), H.host()["val"].tobytes(),
           Eg.cpu().numpy().tobytes(), ag.cpu().numpy().tobytes(), alpha.cpu().numpy().tobytes())
    assert cs.status()["flags"] == 0
    ref = _step(_contact_scene(b, (b.body, b.n_scenes)), b, t1)
    want = (np.array([ref["E"]]).tobytes(), ref["g"].tobytes(), ref["H"]["val"].tobytes(), ref["Eg"].tobytes(),
            ref["ag"].tobytes(), np.array([ref["alpha"]]).tobytes())
    assert got == want


def test_launch_shape_does_not_change_results():
    b = _batch()
    outs = []
    for shape in [None, ("eval_barrier", 64, 8, 3), ("eval_barrier", 128, 2, 2), ("eval_barrier", 128, 4, 4),
                  ("bvh_query", 256, 4, 2), ("bvh_query", 64, 32, 2), ("bvh_query", 256, 6, 3),
                  ("bvh_refit", 256, 8, 0), ("bvh_refit", 256, 8, 1), ("eval_tile", 256, 1, 0),
                  ("eval_tile", 64, 1, 0), ("ccd_tile", 32, 1, 0), ("ccd_tile", 256, 1, 0)]:
        cs = _contact_scene(b, (b.body, b.n_scenes))
        if shape is not None:
            cs.set_launch(*shape)
        r = _step(cs, b, 9)
        outs.append((r["g"].tobytes(), r["H"]["val"].tobytes(), r["Eg"].tobytes(), r["ag"].tobytes()))
    assert all(o == outs[0] for o in outs)


def test_set_groups_rejects_a_primitive_across_groups():
    b = _batch()
    cs = _contact_scene(b)
    bad = b.body.copy()
    v0, nv = b.vertex_ranges[1]
    bad[v0] = 0                                  # one vertex of scene 1 moved to scene 0
    with pytest.raises(RuntimeError):
        cs.set_groups(bad, b.n_scenes)
    with pytest.raises(RuntimeError):
        cs.set_groups(b.body, 1)                 # ids out of range
