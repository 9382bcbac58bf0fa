"""Scene-level pins of the oracle: contact-set enumeration, reduction through the
embedding (Eq. 17: grad_q = J^T grad_x, hess_q = J^T hess_x J), its special cases
(identity embedding = full-space IPC), invariances, and the CCD step bound."""
import functools

import numpy as np

import oracle
from paper_2409_16385_gb300 import scenes


@functools.lru_cache(maxsize=None)
def _scene(k, small=True):
    return scenes.make_config(k, small=small)


def _dense_J(sc):
    """J = d phi / d q as a dense (3 Nv x 3 Ns) matrix (Sec. III-D)."""
    J = np.zeros((3 * sc.Nv, 3 * sc.Ns))
    for v in range(sc.Nv):
        if sc.cage_idx[v, 0] < 0:
            continue
        for j in range(4):
            for k in range(3):
                J[3 * v + k, 3 * sc.cage_idx[v, j] + k] += sc.w[v, j]
    return J


def _stencil(sc, t, i, j):
    if t == 0:
        return np.array([i, *sc.tris[j]])
    return np.array([*sc.edges[i], *sc.edges[j]])


def _dense_blocks(res, ns):
    H = np.zeros((3 * ns, 3 * ns))
    for I, J, V in zip(res["I"], res["J"], res["V"]):
        H[3 * I:3 * I + 3, 3 * J:3 * J + 3] = V
    return H


def test_embedding_reproduces_rest_positions():
    sc = _scene(1)
    x = oracle.embed(sc, sc.q_rest)
    emb = ~sc.kinematic
    assert np.allclose(sc.w[emb].sum(1), 1.0, atol=1e-14)
    assert np.all(sc.w[emb] >= -1e-12)
    r = np.linalg.norm(x[emb], axis=1)
    assert np.allclose(r, 0.05, rtol=1e-12)      # icosphere vertices on the sphere
    assert np.allclose(x @ np.eye(3), oracle.embed(sc, sc.q_rest))
    J = _dense_J(sc)
    q = sc.iterate(0)
    assert np.allclose(oracle.embed(sc, q)[emb].ravel(), (J @ q.ravel()).reshape(-1, 3)[emb].ravel(), atol=1e-15)


def _check_reduction(sc, q, lag_q=None):
    x = oracle.embed(sc, q)
    prs = oracle.pairs(sc, x)
    assert len(prs["type"]) > 0
    lag = None
    if lag_q is not None:
        xn = oracle.embed(sc, lag_q)
        lag = oracle.friction_lag(sc, xn, oracle.pairs(sc, xn))
    res = oracle.eval_contact(sc, x, prs, lag)
    # dense full-space assembly from the per-pair local outputs, then J^T . J
    p = sc.params
    gx = np.zeros(3 * sc.Nv); Hx = np.zeros((3 * sc.Nv, 3 * sc.Nv)); Etot = 0.0
    for t, i, j in zip(prs["type"], prs["i"], prs["j"]):
        s = _stencil(sc, t, i, j)
        E, g, H, Hp = oracle.pair_barrier(t, x[s].ravel(), p["dhat"], p["kappa"])
        Etot += E
        dof = (3 * s[:, None] + np.arange(3)).ravel()
        gx[dof] += g
        Hx[np.ix_(dof, dof)] += Hp
    if lag is not None:
        eps = p["eps_v"] * p["h"]
        for f in range(len(lag["lam"])):
            s = lag["v"][f]
            E, g, H = oracle.pair_friction(s, lag["gamma"][f], lag["n"][f], lag["anchor"][f], lag["lam"][f],
                                           x[s].ravel(), p["mu"], eps)
            Etot += E
            dof = (3 * s[:, None] + np.arange(3)).ravel()
            gx[dof] += g
            Hx[np.ix_(dof, dof)] += H
    J = _dense_J(sc)
    assert np.isclose(res["E"], Etot, rtol=1e-13)
    gr = J.T @ gx
    assert np.abs(res["g"].ravel() - gr).max() <= 1e-12 * np.abs(gr).max()
    Hr = J.T @ Hx @ J
    Hd = _dense_blocks(res, sc.Ns)
    assert np.abs(Hd - Hr).max() <= 1e-12 * np.abs(Hr).max()
    return res, Hd, x, prs, lag


def test_reduction_equals_dense_JT_H_J_config1():
    sc = _scene(1)
    _check_reduction(sc, sc.iterate(0), lag_q=sc.iterate(0))


def test_reduction_equals_dense_JT_H_J_config2_small():
    sc = _scene(2)
    _check_reduction(sc, sc.iterate(4), lag_q=sc.iterate(3))


def test_reduced_invariants_all_embedded():
    """Config 2 has no kinematic vertex: the barrier is invariant to rigid motion of q,
    so sum_I g_I = 0, sum_I q_I x g_I = 0 and H_r annihilates rigid translations; the
    projected H_r is symmetric PSD."""
    sc = _scene(2)
    q = sc.iterate(5)
    x = oracle.embed(sc, q)
    prs = oracle.pairs(sc, x)
    res = oracle.eval_contact(sc, x, prs, None)
    g = res["g"]
    scale = np.abs(g).max()
    assert np.abs(g.sum(0)).max() <= 1e-10 * scale
    assert np.abs(np.cross(q, g).sum(0)).max() <= 1e-9 * scale * np.abs(q).max()
    H = _dense_blocks(res, sc.Ns)
    hs = np.abs(H).max()
    assert np.abs(H - H.T).max() <= 1e-14 * hs
    for k in range(3):
        tvec = np.zeros((sc.Ns, 3)); tvec[:, k] = 1.0
        assert np.abs(H @ tvec.ravel()).max() <= 1e-10 * hs
    nz = np.unique(np.concatenate([res["I"], res["J"]]))
    dof = (3 * nz[:, None] + np.arange(3)).ravel()
    assert np.linalg.eigvalsh(H[np.ix_(dof, dof)]).min() >= -1e-10 * hs


def test_identity_embedding_is_full_space_ipc():
    """phi = identity (each vertex its own node, Sec. III-D last paragraph): the reduced
    gradient and Hessian are the full-space IPC ones."""
    base = _scene(1)
    sc = scenes.Scene(**{f.name: getattr(base, f.name) for f in scenes.dataclasses.fields(base)})
    x = oracle.embed(base, base.iterate(0))
    sc.Ns = base.Nv
    sc.cage_idx = np.repeat(np.arange(base.Nv, dtype=np.int32)[:, None], 4, 1)
    sc.cage_idx[base.kinematic] = -1
    sc.w = np.zeros((base.Nv, 4)); sc.w[:, 0] = 1.0
    sc.w[base.kinematic] = 0.0
    q = x.copy()
    x_id = oracle.embed(sc, q)
    assert np.array_equal(x_id, x)
    prs = oracle.pairs(sc, x)
    res = oracle.eval_contact(sc, x, prs, None)
    p = sc.params
    gx = np.zeros((sc.Nv, 3))
    for t, i, j in zip(prs["type"], prs["i"], prs["j"]):
        s = _stencil(sc, t, i, j)
        _, g, _, _ = oracle.pair_barrier(t, x[s].ravel(), p["dhat"], p["kappa"])
        gx[s] += g.reshape(4, 3)
    gx[base.kinematic] = 0
    assert np.abs(res["g"] - gx).max() <= 1e-12 * np.abs(gx).max()


def test_reduced_gradient_and_hessian_vs_finite_differences():
    """E(q) through the embedding: g_r is its gradient and the unprojected H_r its
    Hessian, checked by central differences in q (contact set held fixed)."""
    sc = _scene(1)
    q0 = sc.iterate(0)
    x = oracle.embed(sc, q0)
    prs = oracle.pairs(sc, x)
    res = oracle.eval_contact(sc, x, prs, None, project=False)
    nodes = np.unique(res["I"])[:6]
    h = 1e-8
    H = _dense_blocks(res, sc.Ns)
    for I in nodes:
        for k in range(3):
            e = np.zeros_like(q0); e[I, k] = h
            rp = oracle.eval_contact(sc, oracle.embed(sc, q0 + e), prs, None, project=False)
            rm = oracle.eval_contact(sc, oracle.embed(sc, q0 - e), prs, None, project=False)
            fd = (rp["E"] - rm["E"]) / (2 * h)
            assert np.isclose(res["g"][I, k], fd, rtol=1e-6, atol=1e-6 * np.abs(res["g"]).max())
            col = (rp["g"] - rm["g"]).ravel() / (2 * h)
            assert np.abs(H[:, 3 * I + k] - col).max() <= 2e-5 * np.abs(H).max()


def test_pair_set_properties_config1():
    sc = _scene(1)
    x = oracle.embed(sc, sc.iterate(0))
    prs = oracle.pairs(sc, x)
    dhat = sc.params["dhat"]
    assert np.all((prs["d"] > 0) & (prs["d"] < dhat))
    key = prs["type"].astype(np.int64) << 52 | prs["i"].astype(np.int64) << 26 | prs["j"].astype(np.int64)
    assert np.all(np.diff(key) > 0)                  # canonical order, no duplicates
    kin = sc.kinematic
    for t, i, j in zip(prs["type"], prs["i"], prs["j"]):
        s = _stencil(sc, t, i, j)
        assert len(set(s.tolist())) == 4             # not incident
        assert not kin[s].all()
    assert np.all(prs["i"][prs["type"] == 1] < prs["j"][prs["type"] == 1])
    # every PT pair of a sampled vertex agrees with the query-restricted enumeration
    for v in np.unique(prs["i"][prs["type"] == 0])[:5]:
        sub = oracle.pairs_of(sc, x, 0, np.array([v]))
        m = (prs["type"] == 0) & (prs["i"] == v)
        assert np.array_equal(sub["j"], prs["j"][m])


def test_pair_set_known_configuration():
    """Two triangles facing each other at a known gap: exactly the expected pairs."""
    gap = 4e-4
    verts = np.array([[0, 0, 0], [1e-2, 0, 0], [0, 1e-2, 0],
                      [2e-3, 2e-3, gap], [6e-3, 2e-3, gap], [2e-3, 6e-3, gap]], float)
    tris = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    sc = scenes.Scene(name="two_tris", tris=tris, edges=scenes.edges_of(tris),
                      cage_idx=np.full((6, 4), -1, np.int32), w=np.zeros((6, 4)), x_kin=verts, Ns=0,
                      cage_tets=np.zeros((0, 4), np.int32), q_rest=np.zeros((0, 3)), body=np.zeros(6, np.int32),
                      params=dict(scenes.DEFAULT_PARAMS))
    sc.cage_idx[3:, :] = 0   # not all-kinematic; weights irrelevant for enumeration
    prs = oracle.pairs(sc, verts)
    pt = sorted(zip(prs["i"][prs["type"] == 0].tolist(), prs["j"][prs["type"] == 0].tolist()))
    assert pt == [(3, 0), (4, 0), (5, 0)]     # upper vertices over the lower face
    assert np.allclose(prs["d"][prs["type"] == 0], gap)
    # EE: every upper edge is farther than dhat from every lower edge
    assert (prs["type"] == 1).sum() == 0


def test_friction_lag_is_the_lagged_contact_force():
    """The lagged state of Sec. III-B, pinned to the per-pair barrier gradient: lambda is the
    magnitude of the contact force at x^n, i.e. of the barrier gradient summed over one side
    of the pair (moving a side rigidly by delta changes d by n . delta); n is the direction in
    which that side's distance grows; the anchor joins the closest points, so its length is
    the pair distance; gamma holds barycentric weights of the closest points, nonnegative
    and summing to 1 on side A, to -1 on side B."""
    sc = _scene(1)
    p = sc.params
    x = oracle.embed(sc, sc.iterate(0))
    prs = oracle.pairs(sc, x)
    lag = oracle.friction_lag(sc, x, prs)
    n_pairs = len(prs["type"])
    assert n_pairs > 20
    for k in range(0, n_pairs, max(1, n_pairs // 200)):
        t, i, j = prs["type"][k], prs["i"][k], prs["j"][k]
        s = _stencil(sc, t, i, j)
        assert np.array_equal(lag["v"][k], s)
        _, g, _, _ = oracle.pair_barrier(t, x[s].ravel(), p["dhat"], p["kappa"])
        side_a = 1 if t == 0 else 2
        force = g.reshape(4, 3)[:side_a].sum(0)
        fn = np.linalg.norm(force)
        assert abs(lag["lam"][k] - fn) <= 1e-10 * fn
        n = lag["n"][k]
        assert abs(np.linalg.norm(n) - 1.0) <= 1e-14
        assert n @ force <= -(1.0 - 1e-9) * fn          # b' < 0: the force pushes along n
        assert abs(np.linalg.norm(lag["anchor"][k]) - prs["d"][k]) <= 1e-12 * prs["d"][k]
        gam = lag["gamma"][k]
        assert np.all(gam[:side_a] >= -1e-15) and np.all(gam[side_a:] <= 1e-15)
        assert abs(gam[:side_a].sum() - 1.0) <= 1e-14 and abs(gam[side_a:].sum() + 1.0) <= 1e-14


# ----------------------------------------------------------------------- CCD step bound

def test_ca_point_plane_constant_velocity():
    """Point falling on a large triangle at speed v from d0: t* = d0/v.  With the mean
    displacement removed L = v, so one advancement lands at (1-s) t*, where d = s d0."""
    T = np.array([[-1.0, -1.0, 0.0], [2.0, -1.0, 0.0], [-1.0, 2.0, 0.0]])
    for d0, v in [(1e-3, 5e-3), (2e-4, 1e-2), (1e-3, 1e-3)]:
        p = np.array([0.1, 0.2, d0])
        x4 = np.concatenate([p, T.ravel()])
        dx4 = np.zeros(12); dx4[2] = -v
        t, it, cap = oracle.ca_pair(0, x4, dx4, s=0.1)
        tstar = d0 / v
        if tstar >= 1.0 / 0.9:
            assert t == 1.0
        else:
            # d(t) = d0 - v t exactly; rounding decides whether the first landing point
            # already satisfies d <= s d0 (one step) or needs one more (t = 0.99 t*)
            assert (1 - 0.1) * tstar * (1 - 1e-12) <= t <= tstar
            assert it <= 2 and (np.isclose(t, 0.9 * tstar, rtol=1e-12) or np.isclose(t, 0.99 * tstar, rtol=1e-12))


def test_ca_advances_by_the_speed_bound_until_s_d0():
    """A point sliding while it falls onto a large triangle: the advancement's speed bound L
    (Sec. III-C; with the mean displacement removed, L = |dx| of the point) exceeds the
    closing speed v, so each advance closes the fraction (1 - s) v / L of the distance:
    d_k = d0 r^k with r = 1 - (1 - s) v / L, and t_k = (1 - s) (d0 / L) (1 - r^k) / (1 - r).
    The advancement stops at the first k with d_k <= s d0.  The numbers put r^2 at 0.075,
    well between s/2 and s, so the count and the time are fixed by the stopping rule."""
    T = np.array([[-1.0, -1.0, 0.0], [2.0, -1.0, 0.0], [-1.0, 2.0, 0.0]])
    s, d0, v = 0.1, 1e-3, 5e-3
    r = np.sqrt(0.075)
    L = (1 - s) * v / (1 - r)
    a = np.sqrt(L * L - v * v)                 # tangential speed
    x4 = np.concatenate([[0.1, 0.2, d0], T.ravel()])
    dx4 = np.zeros(12); dx4[0] = a; dx4[2] = -v
    t, it, cap = oracle.ca_pair(0, x4, dx4, s=s)
    k = 2                                      # r = 0.274 > s >= r^2 = 0.075 > s / 2
    assert r > s >= r ** k > s / 2
    assert it == k and not cap
    assert np.isclose(t, (1 - s) * d0 / L * (1 - r ** k) / (1 - r), rtol=1e-12)


def test_ca_separating_and_edges():
    T = np.array([[-1.0, -1.0, 0.0], [2.0, -1.0, 0.0], [-1.0, 2.0, 0.0]])
    x4 = np.concatenate([[0.1, 0.2, 1e-3], T.ravel()])
    dx4 = np.zeros(12); dx4[2] = +1e-2
    assert oracle.ca_pair(0, x4, dx4)[0] == 1.0
    # crossing edges closing at relative speed v: contact at t* = gap / v
    gap, v = 1e-3, 4e-3
    x4 = np.array([-1, 0, 0, 1, 0, 0, 0, -1, gap, 0, 1, gap], float)
    dx4 = np.array([0, 0, v / 2, 0, 0, v / 2, 0, 0, -v / 2, 0, 0, -v / 2], float)
    t, it, _ = oracle.ca_pair(1, x4, dx4, s=0.1)
    assert t <= gap / v and t >= 0.9 * gap / v * (1 - 1e-12)
    # tangential sliding at constant gap never stops the step
    dx4 = np.array([0.5, 0, 0, 0.5, 0, 0, 0, 0, 0, 0, 0, 0], float)
    assert oracle.ca_pair(1, x4, dx4)[0] == 1.0


def test_ca_bound_depends_only_on_relative_motion():
    """Advancement removes the stencil's mean displacement (Sec. III-C, the accumulated CCD
    reading), so a common translation added to all four displacements leaves the bound
    unchanged up to rounding, however large it is."""
    r = np.random.default_rng(5)
    T = np.array([[-1.0, -1.0, 0.0], [2.0, -1.0, 0.0], [-1.0, 2.0, 0.0]]) * 1e-2
    stopped = 0
    for trial in range(30):
        ptype = trial % 2
        if ptype == 0:
            x4 = np.concatenate([[1e-3, 2e-3, 1e-3], T.ravel()])
        else:
            gap = 1e-3
            x4 = np.array([-1e-2, 0, 0, 1e-2, 0, 0, 0, -1e-2, gap, 0, 1e-2, gap], float)
        dx4 = r.normal(size=12) * 1e-3
        # side A closes on side B along z at 2e-3 per unit step, plus random relative motion
        dx4[2::3] += (np.array([1.0, 1.0, -1.0, -1.0]) if ptype else np.array([-1.0, 0.0, 0.0, 0.0])) * 2e-3
        t0 = oracle.ca_pair(ptype, x4, dx4, s=0.1)[0]
        u = r.normal(size=3) * 5e-2
        t1 = oracle.ca_pair(ptype, x4, dx4 + np.tile(u, 4), s=0.1)[0]
        assert abs(t1 - t0) <= 1e-9 * t0, (trial, t0, t1)
        stopped += t0 < 1.0
    assert stopped >= 20


def _sheets(n=4, gap=1e-3, seed=0):
    """Two n x n vertex grids of triangles, the lower one kinematic, the upper one closing
    on it by twice the gap with a random jitter per vertex."""
    r = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 2) * 2e-3
    lo = np.concatenate([g, np.zeros((n * n, 1))], 1)
    hi = np.concatenate([g + 7e-4, np.full((n * n, 1), gap)], 1)
    quads = [(i * n + j, (i + 1) * n + j, i * n + j + 1, (i + 1) * n + j + 1)
             for i in range(n - 1) for j in range(n - 1)]
    tri = np.array([t for a, b, c, d in quads for t in ((a, b, c), (b, d, c))], np.int32)
    tris = np.concatenate([tri, tri + n * n]).astype(np.int32)
    V = np.concatenate([lo, hi])
    nv = len(V)
    cage_idx = np.full((nv, 4), -1, np.int32)
    cage_idx[n * n:] = 0
    sc = scenes.Scene(name="sheets", tris=tris, edges=scenes.edges_of(tris), cage_idx=cage_idx,
                      w=np.zeros((nv, 4)), x_kin=V, Ns=1, cage_tets=np.zeros((0, 4), np.int32),
                      q_rest=np.zeros((1, 3)), body=np.zeros(nv, np.int32), params=dict(scenes.DEFAULT_PARAMS))
    dx = np.zeros_like(V)
    dx[n * n:] = r.normal(size=(n * n, 3)) * 3e-4 + np.array([0.0, 0.0, -2.0 * gap])
    return sc, V, dx


def _swept_candidates(sc, x, dx):
    """Every non-incident, not all-kinematic PT and EE pair whose swept boxes (over the
    start and end positions of its vertices) overlap, by brute force."""
    x1 = x + dx
    kin = sc.kinematic

    def boxes(ids):
        pts = np.concatenate([x[ids], x1[ids]], axis=1)
        return pts.min(1), pts.max(1)

    vlo, vhi = boxes(np.arange(sc.Nv)[:, None])
    flo, fhi = boxes(sc.tris)
    elo, ehi = boxes(sc.edges)
    out = {"type": [], "i": [], "j": []}
    for v in range(sc.Nv):
        for f in range(sc.F):
            st = np.array([v, *sc.tris[f]])
            if v in sc.tris[f] or kin[st].all():
                continue
            if np.all(vlo[v] <= fhi[f]) and np.all(flo[f] <= vhi[v]):
                out["type"].append(0); out["i"].append(v); out["j"].append(f)
    for e in range(sc.E):
        for g in range(e + 1, sc.E):
            st = np.array([*sc.edges[e], *sc.edges[g]])
            if len(set(st.tolist())) < 4 or kin[st].all():
                continue
            if np.all(elo[e] <= ehi[g]) and np.all(elo[g] <= ehi[e]):
                out["type"].append(1); out["i"].append(e); out["j"].append(g)
    return {k: np.array(v, np.int32) for k, v in out.items()}


def test_restricted_step_bounds_match_the_full_one():
    """The sampled forms of the step bound: over a brute-force list of the swept-box
    candidates, and over the pairs of given query primitives, they reach the full bound
    exactly (the same pairs advanced the same way)."""
    sc, x, dx = _sheets()
    full = oracle.accd(sc, x, dx)
    assert 0.0 < full["alpha"] < 1.0
    cand = _swept_candidates(sc, x, dx)
    assert full["n_candidates"] == len(cand["type"])
    assert oracle.accd_list(sc, x, dx, cand)["alpha"] == full["alpha"]
    a_v = oracle.accd_of(sc, x, dx, 0, np.arange(sc.Nv))
    a_e = oracle.accd_of(sc, x, dx, 1, np.arange(sc.E))
    assert min(a_v["alpha"], a_e["alpha"]) == full["alpha"]
    n_pt = int((cand["type"] == 0).sum())
    assert a_v["n_candidates"] == n_pt and a_e["n_candidates"] == 2 * (len(cand["type"]) - n_pt)
    # a subset of queries never bounds the step more tightly than all of them
    assert oracle.accd_of(sc, x, dx, 1, np.arange(0, sc.E, 3))["alpha"] >= full["alpha"]


def test_restricted_edge_pairs_match_the_full_set():
    """EE pairs of sampled edges are exactly the full set's EE pairs that have one of those
    edges as a side, in (i, j) order with i < j; a pair with both sides among the queries
    is listed once per side."""
    sc = _scene(1)
    x = oracle.embed(sc, sc.iterate(0))
    prs = oracle.pairs(sc, x)
    ee = np.nonzero(prs["type"] == 1)[0]
    i, j, d = prs["i"][ee], prs["j"][ee], prs["d"][ee]
    q = np.unique(np.concatenate([i[:6], j[-6:], [j[0], 0, 17]]))
    sub = oracle.pairs_of(sc, x, 1, q)
    times = np.isin(i, q).astype(int) + np.isin(j, q).astype(int)
    assert (times > 0).sum() > 6 and (times == 2).any()
    assert np.array_equal(sub["i"], np.repeat(i, times)) and np.array_equal(sub["j"], np.repeat(j, times))
    assert np.array_equal(sub["d"], np.repeat(d, times))


def test_ca_iteration_cap_returns_safe_time():
    T = np.array([[-1.0, -1.0, 0.0], [2.0, -1.0, 0.0], [-1.0, 2.0, 0.0]])
    x4 = np.concatenate([[0.1, 0.2, 1e-3], T.ravel()])
    dx4 = np.zeros(12); dx4[2] = -1.0; dx4[0] = 50.0
    t, it, cap = oracle.ca_pair(0, x4, dx4, s=0.1, max_iter=1)
    assert cap and it == 1 and 0 < t < 1e-3


def test_accd_no_penetration_after_accepted_step_config1():
    """Step bound on the sphere-on-pad scene: positions at alpha (and the accepted 0.9
    alpha) are intersection-free; the full step is not (the check has teeth)."""
    sc = _scene(1)
    q = sc.iterate(0)
    x = oracle.embed(sc, q)
    dx = oracle.embed(sc, sc.dq(0), displacement=True)
    r = oracle.accd(sc, x, dx)
    a = r["alpha"]
    assert 0 < a < 1 and r["n_candidates"] > 0 and not r["capped"]
    assert oracle.intersection_free(sc, x)
    assert oracle.intersection_free(sc, x + a * dx)
    assert oracle.intersection_free(sc, x + 0.9 * a * dx)
    assert not oracle.intersection_free(sc, x + dx)
    # linearity of phi: the bound along J dq equals the bound along J dq1 + J dq2
    dq1 = 0.3 * sc.dq(0); dq2 = sc.dq(0) - dq1
    dx12 = oracle.embed(sc, dq1, displacement=True) + oracle.embed(sc, dq2, displacement=True)
    assert np.allclose(dx12, dx, atol=1e-18)


def test_trajectories_are_intersection_free_small():
    for k in (2, 3):
        sc = _scene(k)
        for t in (0, sc.n_iterates // 2, sc.n_iterates - 1):
            x = oracle.embed(sc, sc.iterate(t))
            assert oracle.intersection_free(sc, x)
            prs = oracle.pairs(sc, x)       # raises on d <= 0
            assert len(prs["type"]) > 0
