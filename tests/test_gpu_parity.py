"""GPU parity: the CUDA contact stage (through the C ABI) against the CPU oracle, element
by element on the same seeded inputs.

Bars (all stated against the oracle's values):
  contact set   identical (type, i, j) lists, except pairs with |d - dhat| <= 1e-12 dhat;
                d within 1e-10 relative
  E             |dE| <= 1e-9 |E|
  g_r           max |dg| <= 1e-9 max |g|
  H_r           identical block pattern, max |dH| <= 1e-9 max |H|
  alpha         alpha_gpu <= alpha_oracle and alpha_oracle - alpha_gpu <= 1e-6
"""
import functools

import numpy as np
import pytest

import oracle
from paper_2409_16385_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-9


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@functools.lru_cache(maxsize=None)
def _scene(k, small):
    return scenes.make_config(k, small=small)


_cs_cache = {}


def _cs(sc):
    from paper_2409_16385_gb300 import ContactScene
    key = id(sc)
    if key not in _cs_cache:
        _cs_cache[key] = ContactScene(sc, pair_capacity=1 << 20, bsr_capacity=1 << 21)
    return _cs_cache[key]


def check_pairs(g, o, dhat):
    kg = list(zip(g["type"].tolist(), g["i"].tolist(), g["j"].tolist()))
    ko = list(zip(o["type"].tolist(), o["i"].tolist(), o["j"].tolist()))
    assert kg == sorted(kg), "GPU pair list not in (type, i, j) order"
    sg, so = set(kg), set(ko)
    dg = dict(zip(kg, g["d"].tolist()))
    do = dict(zip(ko, o["d"].tolist()))
    for k in sg ^ so:
        d = dg.get(k, do.get(k))
        assert abs(d - dhat) <= 1e-12 * dhat, f"pair {k} (d={d!r}) differs outside the dhat band"
    common = sg & so
    if common:
        err = max(abs(dg[k] - do[k]) / do[k] for k in common)
        assert err <= 1e-10, err
    return len(common)


def bsr_dict(H, ns):
    rp, col, val = H["row_ptr"], H["col"], H["val"]
    out = {}
    for r in range(ns):
        for k in range(rp[r], rp[r + 1]):
            out[(r, int(col[k]))] = val[k]
    return out


def check_eval(E, g, H, ro, ns):
    Eg = float(E)
    assert abs(Eg - ro["E"]) <= TOL * abs(ro["E"]) + 1e-300, (Eg, ro["E"])
    gs = np.abs(ro["g"]).max()
    assert np.abs(g - ro["g"]).max() <= TOL * gs + 1e-300
    hg = bsr_dict(H, ns)
    ho = {(int(i), int(j)): v for i, j, v in zip(ro["I"], ro["J"], ro["V"])}
    assert set(hg) == set(ho), "reduced Hessian block patterns differ"
    hs = max((np.abs(v).max() for v in ho.values()), default=0.0)
    err = max((np.abs(hg[k] - ho[k]).max() for k in ho), default=0.0)
    assert err <= TOL * hs + 1e-300, (err, hs)
    # rows sorted, full symmetric pattern
    rp, col = H["row_ptr"], H["col"]
    for r in range(ns):
        assert np.all(np.diff(col[rp[r]:rp[r + 1]]) > 0)
    return err / hs if hs else 0.0


def run_iterate(sc, t, lag_t=None, check_alpha=True):
    """Full pipeline at iterate t on both sides; returns the GPU outputs."""
    cs = _cs(sc)
    p = sc.params
    q = sc.iterate(t)
    lag_t = sc.lag_of(t) if lag_t is None else lag_t
    qn = sc.iterate(lag_t)
    qd, qnd = _t(q), _t(qn)
    # GPU
    pairs_n = cs.build_candidates(qnd, out=cs.new_pairs())
    lag = cs.friction_lag(qnd, pairs_n) if p["mu"] > 0 else None
    pairs = cs.build_candidates(qd)
    E, g, H = cs.eval_contact(qd, pairs, lag)
    torch.cuda.synchronize()
    st = cs.status()
    assert st["flags"] == 0, st
    # oracle
    x, xn = oracle.embed(sc, q), oracle.embed(sc, qn)
    po, pon = oracle.pairs(sc, x), oracle.pairs(sc, xn)
    lo = oracle.friction_lag(sc, xn, pon) if p["mu"] > 0 else None
    ro = oracle.eval_contact(sc, x, po, lo)
    ncommon = check_pairs(pairs.host(), po, p["dhat"])
    check_pairs(pairs_n.host(), pon, p["dhat"])
    if lo is not None:
        lg = lag.host()
        assert len(lg["lam"]) == len(lo["lam"])
        assert np.array_equal(lg["v"], lo["v"])
        assert np.allclose(lg["lam"], lo["lam"], rtol=1e-9, atol=0)
        assert np.allclose(lg["gamma"], lo["gamma"], atol=1e-9)
        assert np.allclose(lg["n"], lo["n"], atol=1e-9)
    rel = check_eval(E.item(), g.cpu().numpy(), H.host(), ro, sc.Ns)
    alpha = None
    if check_alpha:
        dq = sc.dq(t)
        xg = cs.embed(qd)
        dxg = cs.embed(_t(dq), displacement=True)
        a = cs.accd_toi(xg, dxg).item()
        ao = oracle.accd(sc, x, oracle.embed(sc, dq, displacement=True))
        assert a <= ao["alpha"], (a, ao)
        assert ao["alpha"] - a <= 1e-6, (a, ao)
        alpha = (a, ao["alpha"])
        assert cs.status()["flags"] == 0
    return dict(pairs=ncommon, rel=rel, alpha=alpha, E=ro["E"])


def test_config1_sphere_on_pad():
    sc = _scene(1, False)
    r = run_iterate(sc, 0)
    assert r["pairs"] > 100 and 0 < r["alpha"][1] < 1
    # second evaluation at q0 + alpha/2 dq: friction now sees tangential motion
    sc2 = scenes.with_second_iterate(sc, r["alpha"][1])
    r2 = run_iterate(sc2, 1, lag_t=0, check_alpha=False)
    assert r2["pairs"] > 0


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("t", [0, 7, 13])
def test_small_trajectories(k, t):
    sc = _scene(k, True)
    t = min(t, sc.n_iterates - 2)
    r = run_iterate(sc, t)
    assert r["pairs"] > 0


@pytest.mark.parametrize("k,t", [(2, 30), (3, 40)])
def test_full_size_iterate(k, t):
    """Benchmark-size scenes, whole outputs (the oracle enumerates all pairs)."""
    oracle.set_threads(max(1, oracle.num_threads()))
    sc = _scene(k, False)
    r = run_iterate(sc, t)
    assert r["pairs"] > 1000


def test_bitwise_repeatable():
    sc = _scene(2, True)
    cs = _cs(sc)
    q = _t(sc.iterate(9))
    qn = _t(sc.iterate(sc.lag_of(9)))
    lag = cs.friction_lag(qn, cs.build_candidates(qn, out=cs.new_pairs()))
    outs = []
    for _ in range(3):
        pr = cs.build_candidates(q)
        E, g, H = cs.eval_contact(q, pr, lag)
        h = H.host()
        outs.append((E.cpu().numpy().tobytes(), g.cpu().numpy().tobytes(), h["val"].tobytes(), h["col"].tobytes()))
    assert outs[0] == outs[1] == outs[2]


def test_launch_modes_agree_bitwise():
    """Programmatic dependent launch (the default) and plain stream order give the same
    bits for the pair set, E, g_r, H_r and the CCD step bound."""
    from paper_2409_16385_gb300 import binding
    sc = _scene(2, True)
    cs = _cs(sc)
    q = _t(sc.iterate(9))
    qn = _t(sc.iterate(sc.lag_of(9)))
    dq = _t(sc.dq(9))
    outs = []
    try:
        for on in (False, True, False, True):
            binding.set_programmatic_launch(on)
            lag = cs.friction_lag(qn, cs.build_candidates(qn, out=cs.new_pairs()))
            pr = cs.build_candidates(q)
            E, g, H = cs.eval_contact(q, pr, lag)
            a = cs.accd_toi(cs.embed(q), cs.embed(dq, displacement=True))
            h = H.host()
            ph = pr.host()
            outs.append((ph["i"].tobytes(), ph["j"].tobytes(), ph["d"].tobytes(), E.cpu().numpy().tobytes(),
                         g.cpu().numpy().tobytes(), h["val"].tobytes(), h["col"].tobytes(), float(a)))
            assert cs.status()["flags"] == 0
    finally:
        binding.set_programmatic_launch(True)
    assert outs[0] == outs[1] == outs[2] == outs[3]


def test_friction_match_by_key_and_by_stencil_agree():
    """A lag state built by the scene is matched to the contact pairs by its recorded pair
    keys; a copy of it in other buffers (no keys) by the stencils' vertices.  The key also
    tells a PT pair from an EE pair with the same four vertices, so it merges at least as
    many items.  Either way E, g_r and H_r are the same sums up to rounding, on the same
    pattern, and each way repeats bitwise."""
    import dataclasses
    sc = _scene(2, True)
    cs = _cs(sc)
    t = 9
    q, qn = _t(sc.iterate(t)), _t(sc.iterate(sc.lag_of(t)))
    lag = cs.friction_lag(qn, cs.build_candidates(qn, out=cs.new_pairs()))
    pr = cs.build_candidates(q)
    copy = dataclasses.replace(lag, **{f.name: getattr(lag, f.name).clone() for f in dataclasses.fields(lag)})
    outs = []
    for lg in (lag, copy, lag, copy):
        E, g, H = cs.eval_contact(q, pr, lg)
        h = H.host()
        outs.append((E.cpu().numpy(), g.cpu().numpy(), h["val"], h["col"], h["row_ptr"],
                     cs.work_counts()["hessian_records"]))
        assert cs.status()["flags"] == 0
    for a, b in ((outs[0], outs[2]), (outs[1], outs[3])):
        assert all(np.array_equal(x, y) for x, y in zip(a[:5], b[:5])) and a[5] == b[5]
    key, vert = outs[0], outs[1]
    assert key[5] <= vert[5]
    assert np.array_equal(key[3], vert[3]) and np.array_equal(key[4], vert[4])
    for x, y in zip(key[:3], vert[:3]):
        assert np.max(np.abs(x - y)) <= 1e-12 * max(np.max(np.abs(y)), 1e-300)


def test_refitted_and_rebuilt_hierarchies_agree_bitwise():
    """The contact set and the reduced outputs do not depend on whether the LBVH was
    rebuilt for these positions or refitted from another configuration's hierarchy."""
    from paper_2409_16385_gb300 import ContactScene
    sc = _scene(2, True)
    a = ContactScene(sc, pair_capacity=1 << 18, bsr_capacity=1 << 18)
    b = ContactScene(sc, pair_capacity=1 << 18, bsr_capacity=1 << 18)
    b.set_rebuild_interval(1)
    a.set_rebuild_interval(1000)
    a.build_candidates(_t(sc.iterate(0)))          # hierarchy from another configuration
    a.build_candidates(_t(sc.iterate(19)))
    q = _t(sc.iterate(11))
    outs = []
    for cs in (a, b):
        pr = cs.build_candidates(q)
        E, g, H = cs.eval_contact(q, pr, None)
        h = H.host()
        ph = pr.host()
        outs.append((ph["type"].tobytes(), ph["i"].tobytes(), ph["j"].tobytes(), ph["d"].tobytes(),
                     E.cpu().numpy().tobytes(), g.cpu().numpy().tobytes(), h["val"].tobytes()))
        assert cs.status()["flags"] == 0
    assert outs[0] == outs[1]


def test_work_counts_match_the_outputs():
    """eipc_work_counts: pairs and items as returned, records recomputed from the stencils'
    cage nodes, and block counts as the BSR pattern shows them."""
    sc = _scene(2, True)
    cs = _cs(sc)
    t = 9
    q, qn = _t(sc.iterate(t)), _t(sc.iterate(sc.lag_of(t)))
    lag = cs.friction_lag(qn, cs.build_candidates(qn, out=cs.new_pairs()))
    pr = cs.build_candidates(q)
    wc_pairs = cs.work_counts()
    E, g, H = cs.eval_contact(q, pr, lag)
    wc = cs.work_counts()
    ph, lh, hh = pr.host(), lag.host(), H.host()
    P, L = len(ph["type"]), len(lh["lam"])
    assert wc_pairs["pairs"] == P and wc["pairs"] == P
    assert wc_pairs["candidates"] >= wc_pairs["screened"] >= P > 0
    assert wc["items"] == P + L
    ci = sc.cage_idx

    def nodes(vs):
        out = []
        for v in vs:
            if ci[v, 0] >= 0:
                out += [n for n in ci[v] if n not in out]
        return len(out)

    st = [tuple(int(a) for a in ([i, *sc.tris[j]] if ty == 0 else [*sc.edges[i], *sc.edges[j]]))
          for ty, i, j in zip(ph["type"], ph["i"], ph["j"])]
    # a friction pair with the stencil of a contact pair (the first such, in lag order)
    # writes into that pair's records
    free, claimed, pairs = [], set(), set(st)
    for v in lh["v"]:
        t = tuple(int(a) for a in v)
        if t in pairs and t not in claimed:
            claimed.add(t)
        else:
            free.append(v)
    assert len(claimed) > 0.5 * L
    ns = [nodes(s) for s in st] + [nodes(v) for v in free]
    assert wc["hessian_records"] == sum(n * (n + 1) // 2 for n in ns)
    assert wc["gradient_records"] == sum(ns)
    rows = np.repeat(np.arange(sc.Ns), np.diff(hh["row_ptr"]))
    n_diag = int(np.sum(rows == hh["col"]))
    assert len(hh["col"]) == 2 * wc["hessian_blocks"] - n_diag
    assert wc["gradient_nodes"] == n_diag
