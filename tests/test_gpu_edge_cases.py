"""GPU edge cases: empty contact set, a touching pair (d = 0), undersized caller buffers,
non-finite input and the CCD iteration cap.  Each condition is reported through the
device status word; none faults the device."""
import numpy as np
import pytest

import oracle
from paper_2409_16385_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _two_triangle_scene(gap):
    """Kinematic triangle at z = 0 and an embedded triangle `gap` above it (each embedded
    vertex is its own cage node)."""
    verts = np.array([[0, 0, 0], [1e-2, 0, 0], [0, 1e-2, 0],
                      [2e-3, 2e-3, gap], [6e-3, 2e-3, gap], [2e-3, 6e-3, gap]], float)
    tris = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    idx = np.full((6, 4), -1, np.int32)
    w = np.zeros((6, 4))
    for v in range(3, 6):
        idx[v] = v - 3
        w[v, 0] = 1.0
    xk = verts.copy(); xk[3:] = 0
    sc = scenes.Scene(name="two_tris", tris=tris, edges=scenes.edges_of(tris), cage_idx=idx, w=w, x_kin=xk, Ns=3,
                      cage_tets=np.zeros((0, 4), np.int32), q_rest=verts[3:].copy(), body=np.array([0, 0, 0, 1, 1, 1], np.int32),
                      params=dict(scenes.DEFAULT_PARAMS))
    return sc, verts[3:].copy()


def test_empty_contact_set():
    from paper_2409_16385_gb300 import ContactScene
    sc, q = _two_triangle_scene(5e-3)          # farther than dhat = 1e-3
    cs = ContactScene(sc, pair_capacity=64, bsr_capacity=64)
    qd = _t(q)
    pr = cs.build_candidates(qd)
    E, g, H = cs.eval_contact(qd, pr, None)
    torch.cuda.synchronize()
    assert pr.n() == 0 and E.item() == 0.0 and float(g.abs().max()) == 0.0
    assert int(H.nnzb.item()) == 0 and int(H.row_ptr.abs().max()) == 0
    assert cs.status()["flags"] == 0
    # three PT pairs at exactly the known gap, and matching the oracle
    sc2, q2 = _two_triangle_scene(4e-4)
    cs2 = ContactScene(sc2, pair_capacity=64, bsr_capacity=64)
    pr2 = cs2.build_candidates(_t(q2)).host()
    x = oracle.embed(sc2, q2)
    po = oracle.pairs(sc2, x)
    assert pr2["type"].tolist() == po["type"].tolist() and pr2["i"].tolist() == po["i"].tolist()
    assert np.allclose(pr2["d"], 4e-4, rtol=1e-12)


def test_touching_pair_raises_penetration_flag():
    from paper_2409_16385_gb300 import ContactScene
    sc, q = _two_triangle_scene(0.0)           # the upper triangle lies in the lower one's plane
    q[:, 2] = 0.0
    q[0] = [2e-3, 2e-3, 0.0]                    # and vertex 3 lies on the lower triangle
    q[1:, 2] = 1e-3
    cs = ContactScene(sc, pair_capacity=64, bsr_capacity=64)
    cs.build_candidates(_t(q))
    torch.cuda.synchronize()
    st = cs.status()
    assert "PENETRATION" in st["names"]
    assert cs.status()["flags"] == 0           # reading clears the word


def test_pair_and_bsr_capacity_overflow_reported():
    from paper_2409_16385_gb300 import ContactScene
    sc = scenes.make_config(1)
    cs = ContactScene(sc, pair_capacity=16, bsr_capacity=8)
    q = _t(sc.iterate(0))
    pr = cs.build_candidates(q)
    torch.cuda.synchronize()
    st = cs.status()
    assert "PAIR_OVERFLOW" in st["names"] and st["needed"][0] > 16
    assert pr.n() == st["needed"][0]           # the true count is still reported
    E, g, H = cs.eval_contact(q, pr, None)
    torch.cuda.synchronize()
    st = cs.status()
    assert "BSR_OVERFLOW" in st["names"] and st["needed"][3] > 8


def test_nonfinite_input_flag():
    from paper_2409_16385_gb300 import ContactScene
    sc = scenes.make_config(1)
    cs = ContactScene(sc, pair_capacity=1 << 12, bsr_capacity=1 << 12)
    q = sc.iterate(0).copy()
    q[sc.cage_idx[0, 0], 1] = np.nan            # a cage node the first surface vertex uses
    cs.build_candidates(_t(q))
    torch.cuda.synchronize()
    assert "NONFINITE" in cs.status()["names"]


def test_accd_iteration_cap_keeps_alpha_safe():
    from paper_2409_16385_gb300 import ContactScene
    sc = scenes.make_config(1)
    sc.params = dict(sc.params, accd_max_iter=1)
    cs = ContactScene(sc, pair_capacity=1 << 12, bsr_capacity=1 << 12)
    q = sc.iterate(0)
    x = cs.embed(_t(q))
    dx = cs.embed(_t(sc.dq(0)), displacement=True)
    a = cs.accd_toi(x, dx).item()
    torch.cuda.synchronize()
    st = cs.status()
    ao = oracle.accd(sc, oracle.embed(sc, q), oracle.embed(sc, sc.dq(0), displacement=True), max_iter=1)
    assert ao["capped"] and "ACCD_CAP" in st["names"]
    assert a <= ao["alpha"] and ao["alpha"] - a <= 1e-6


def _rot(rng):
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return Q


def test_pairs_at_the_dhat_boundary_match_the_oracle():
    """Hundreds of PT (face region) and EE (crossing, down to 1 degree from parallel)
    stencils placed at (1 -+ 1e-4) and (1 -+ 3e-3) dhat: the kept set must be exactly the
    oracle's, whatever shortcuts the narrow phase takes."""
    from paper_2409_16385_gb300 import ContactScene
    rng = np.random.default_rng(11)
    dhat = 1e-3
    verts, tris, emb = [], [], []
    for k in range(240):
        o = np.array([0.02 * (k % 20), 0.02 * (k // 20), 0.0])
        R = _rot(rng)
        rel = [1 - 3e-3, 1 - 1e-4, 1 + 1e-4, 1 + 3e-3][k % 4]
        if k % 2 == 0:
            T = rng.normal(size=(3, 3)) * 2e-3
            T[:, 2] = 0.0
            foot = rng.dirichlet([2, 2, 2]) @ T
            p = foot + np.array([0, 0, rel * dhat])
            up = np.array([p, p + [1e-3, 0, 3e-3], p + [0, 1e-3, 3e-3]])
        else:
            ang = np.radians([1.0, 5.0, 30.0, 90.0][(k // 2) % 4])
            T = np.array([[-1e-3, 0, 0], [1e-3, 0, 0], [0, -1e-3, 0]])
            h = rel * dhat
            dirn = np.array([np.cos(ang), np.sin(ang), 0.0])
            up = np.array([-1e-3 * dirn + [0, 0, h], 1e-3 * dirn + [0, 0, h], [0, 3e-4, h + 2e-3]])
        base = len(verts)
        for v in T:
            verts.append(R @ v + o); emb.append(False)
        for v in up:
            verts.append(R @ v + o); emb.append(True)
        tris += [[base, base + 1, base + 2], [base + 3, base + 4, base + 5]]
    verts = np.array(verts); tris = np.array(tris, np.int32); emb = np.array(emb)
    nv = len(verts)
    idx = np.full((nv, 4), -1, np.int32); w = np.zeros((nv, 4))
    node_of = np.cumsum(emb) - 1
    idx[emb, 0] = node_of[emb]; idx[emb, 1:] = node_of[emb][:, None]
    w[emb, 0] = 1.0
    xk = np.where(emb[:, None], 0.0, verts)
    sc = scenes.Scene(name="boundary", tris=tris, edges=scenes.edges_of(tris), cage_idx=idx, w=w, x_kin=xk,
                      Ns=int(emb.sum()), cage_tets=np.zeros((0, 4), np.int32), q_rest=verts[emb].copy(),
                      body=np.zeros(nv, np.int32), params=dict(scenes.DEFAULT_PARAMS, dhat=dhat))
    q = verts[emb].copy()
    cs = ContactScene(sc, pair_capacity=1 << 14, bsr_capacity=1 << 14)
    g = cs.build_candidates(_t(q)).host()
    torch.cuda.synchronize()
    assert cs.status()["flags"] == 0
    o = oracle.pairs(sc, oracle.embed(sc, q))
    kg = list(zip(g["type"].tolist(), g["i"].tolist(), g["j"].tolist()))
    ko = list(zip(o["type"].tolist(), o["i"].tolist(), o["j"].tolist()))
    assert kg == ko
    near = np.abs(o["d"] / dhat - 1.0) < 5e-3
    assert near.sum() >= 100          # the boundary cases really are in the set


def test_degenerate_surface_primitives_match_the_oracle():
    """A kinematic surface of degenerate triangles (three collinear vertices, two coincident
    vertices, all three coincident) under embedded triangles at 0.3-0.8 dhat.  The
    distance is the minimum over the closed primitive: a collinear triangle is the segment
    it spans, a zero-length edge is its point.  Pair set, distances, E, g_r, H_r and the
    step bound must match the oracle.  The closest-point weights on a degenerate triangle
    are not unique, so friction is off (mu = 0) and only the embedded DoFs carry
    derivatives."""
    from paper_2409_16385_gb300 import ContactScene
    rng = np.random.default_rng(21)
    dhat = 1e-3
    verts, tris, emb = [], [], []
    for k in range(60):
        o = np.array([0.01 * (k % 10), 0.01 * (k // 10), 0.0])
        kind = k % 3
        if kind == 0:          # collinear along x, middle vertex last
            T = np.array([[-1e-3, 0, 0], [1e-3, 0, 0], [rng.uniform(-5e-4, 5e-4), 0, 0]])
        elif kind == 1:        # two coincident vertices: a zero-length edge
            T = np.array([[-1e-3, 0, 0], [1e-3, 0, 0], [1e-3, 0, 0]])
        else:                  # all three coincident
            T = np.zeros((3, 3))
        h = rng.uniform(0.3, 0.8) * dhat
        p = np.array([rng.uniform(-8e-4, 8e-4), rng.uniform(-2e-4, 2e-4), h])
        up = np.array([p, p + [1.5e-3, 2e-4, 2.5e-3], p + [-2e-4, 1.5e-3, 2.5e-3]])
        base = len(verts)
        for v in T:
            verts.append(v + o); emb.append(False)
        for v in up:
            verts.append(v + o); emb.append(True)
        tris += [[base, base + 1, base + 2], [base + 3, base + 4, base + 5]]
    verts = np.array(verts); tris = np.array(tris, np.int32); emb = np.array(emb)
    nv = len(verts)
    idx = np.full((nv, 4), -1, np.int32); w = np.zeros((nv, 4))
    node_of = np.cumsum(emb) - 1
    idx[emb, 0] = node_of[emb]; idx[emb, 1:] = node_of[emb][:, None]
    w[emb, 0] = 1.0
    xk = np.where(emb[:, None], 0.0, verts)
    sc = scenes.Scene(name="degenerate", tris=tris, edges=scenes.edges_of(tris), cage_idx=idx, w=w, x_kin=xk,
                      Ns=int(emb.sum()), cage_tets=np.zeros((0, 4), np.int32), q_rest=verts[emb].copy(),
                      body=np.zeros(nv, np.int32), params=dict(scenes.DEFAULT_PARAMS, dhat=dhat, mu=0.0))
    q = verts[emb].copy()
    dq = np.tile([0.0, 0.0, -1.5e-3], (sc.Ns, 1))
    from test_gpu_parity import check_eval, check_pairs
    cs = ContactScene(sc, pair_capacity=1 << 14, bsr_capacity=1 << 14)
    qd = _t(q)
    pr = cs.build_candidates(qd)
    E, g, H = cs.eval_contact(qd, pr, None)
    x_g = cs.embed(qd)
    dx_g = cs.embed(_t(dq), displacement=True)
    a = cs.accd_toi(x_g, dx_g).item()
    torch.cuda.synchronize()
    assert cs.status()["flags"] == 0
    x = oracle.embed(sc, q)
    po = oracle.pairs(sc, x)
    assert len(po["type"]) >= 60
    assert check_pairs(pr.host(), po, dhat) == len(po["type"])
    ro = oracle.eval_contact(sc, x, po, None)
    check_eval(E.item(), g.cpu().numpy(), H.host(), ro, sc.Ns)
    ao = oracle.accd(sc, x, oracle.embed(sc, dq, displacement=True))["alpha"]
    assert 0.0 < ao < 1.0 and a <= ao and ao - a <= 1e-6


def test_candidate_readout_covers_the_pairs_and_the_ccd_input():
    """eipc_candidates_read returns the broad phase of the last call: after
    build_candidates a superset of the contact pairs; after accd_toi the list whose exact
    FP64 swept-box overlaps are the candidates the CCD advanced, and the oracle's
    advancement over exactly those gives the oracle's step bound."""
    from paper_2409_16385_gb300 import ContactScene
    sc = scenes.make_config(1)
    cs = ContactScene(sc, pair_capacity=1 << 14, bsr_capacity=1 << 16)
    q = sc.iterate(0)
    pairs = cs.build_candidates(_t(q))
    ct, ci, cj = (a.cpu().numpy() for a in cs.candidates())
    h = pairs.host()
    cand = set(zip(ct.tolist(), ci.tolist(), cj.tolist()))
    assert len(h["type"]) > 0
    assert set(zip(h["type"].tolist(), h["i"].tolist(), h["j"].tolist())) <= cand
    x = cs.embed(_t(q))
    dx = cs.embed(_t(sc.dq(0)), displacement=True)
    nadv = torch.zeros(1, dtype=torch.int64, device="cuda")
    a = cs.accd_toi(x, dx, n_candidates=nadv).item()
    ct, ci, cj = (a_.cpu().numpy() for a_ in cs.candidates())
    xo = oracle.embed(sc, q)
    dxo = oracle.embed(sc, sc.dq(0), displacement=True)
    st = np.zeros((len(ct), 4), np.int64)                       # stencil vertices
    pt = ct == 0
    st[pt] = np.c_[ci[pt], sc.tris[cj[pt]]]
    st[~pt] = np.c_[sc.edges[ci[~pt]], sc.edges[cj[~pt]]]
    na = np.where(ct == 0, 1, 2)
    p0, p1 = xo[st], xo[st] + dxo[st]
    lo, hi = np.minimum(p0, p1), np.maximum(p0, p1)
    side_a = np.arange(4)[None, :] < na[:, None]
    big = np.inf
    loA = np.where(side_a[..., None], lo, big).min(1); hiA = np.where(side_a[..., None], hi, -big).max(1)
    loB = np.where(~side_a[..., None], lo, big).min(1); hiB = np.where(~side_a[..., None], hi, -big).max(1)
    ov = ~((loA > hiB) | (loB > hiA)).any(1)
    assert int(ov.sum()) == int(nadv.item())
    ao = oracle.accd(sc, xo, dxo)
    al = oracle.accd_list(sc, xo, dxo, dict(type=ct[ov], i=ci[ov], j=cj[ov]))
    assert al["alpha"] == ao["alpha"]
    assert a <= ao["alpha"] and ao["alpha"] - a <= 1e-6
