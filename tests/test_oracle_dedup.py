"""Pins of the oracle's deduplicated contact set (CPU only).

Hand-built geometry where the answer is fixed by the shapes: a point above the ridge of a
folded pair of triangles is closest to the shared edge from both (one vertex-edge
constraint, not two); a point above the apex of a four-triangle pyramid is closest to the
apex from all four (one vertex-vertex constraint); a point above a face interior keeps its
single face-vertex pair.  On full scenes: the kept pairs realise distinct feature pairs,
every dropped pair realises a kept one, the kept set is a subset in (type, i, j) order,
and the energy does not grow.  Feature pairs are recomputed here from the oracle's region
codes.
"""
import numpy as np
import pytest

import oracle
from paper_2409_16385_gb300 import scenes

DHAT = 1e-3


def _scene(points, surf_v, surf_t):
    """One embedded point cloud (the queries) against a kinematic surface."""
    n_p = len(points)
    V = np.concatenate([points, surf_v]).astype(float)
    tris = (np.asarray(surf_t) + n_p).astype(np.int32)
    cage_idx = np.full((len(V), 4), -1, np.int32)
    cage_idx[:n_p] = [0, 1, 2, 3]
    w = np.zeros((len(V), 4))
    w[:n_p, 0] = 1.0
    x_kin = np.where((cage_idx[:, 0] < 0)[:, None], V, 0.0)
    sc = scenes.Scene(name="hand", tris=tris, edges=scenes.edges_of(tris), cage_idx=cage_idx, w=w, x_kin=x_kin,
                      Ns=4, cage_tets=np.zeros((0, 4), np.int32), q_rest=np.zeros((4, 3)),
                      body=np.zeros(len(V), np.int32), params=dict(scenes.DEFAULT_PARAMS, dhat=DHAT))
    return sc, V


def test_point_above_a_ridge_counts_once():
    h = 0.3 * DHAT
    pts = np.array([[0.5, 0.5, h]])
    surf = np.array([[0, 0, 0], [1, 0, -0.3], [1, 1, 0], [0, 1, -0.3]], float)
    sc, x = _scene(pts, surf, [[0, 1, 2], [0, 2, 3]])
    lit = oracle.pairs(sc, x)
    assert len(lit["type"]) == 2 and np.all(lit["type"] == 0)
    dd = oracle.dedup(sc, x, lit)
    assert len(dd["type"]) == 1 and (dd["type"][0], dd["i"][0], dd["j"][0]) == (0, lit["i"][0], lit["j"][0])
    e_lit = oracle.eval_contact(sc, x, lit, None)["E"]
    e_dd = oracle.eval_contact(sc, x, dd, None)["E"]
    assert abs(e_lit - 2 * e_dd) <= 1e-12 * e_lit


def test_point_above_a_pyramid_apex_counts_once():
    h = 0.4 * DHAT
    pts = np.array([[0.0, 0.0, h]])
    surf = np.array([[0, 0, 0], [1, 0, -1], [0, 1, -1], [-1, 0, -1], [0, -1, -1]], float)
    sc, x = _scene(pts, surf, [[0, 1, 2], [0, 2, 3], [0, 3, 4], [0, 4, 1]])
    lit = oracle.pairs(sc, x)
    assert len(lit["type"]) == 4
    dd = oracle.dedup(sc, x, lit)
    assert len(dd["type"]) == 1
    assert abs(dd["d"][0] - h) <= 1e-15


def test_point_above_a_face_interior_is_kept():
    pts = np.array([[0.3, 0.3, 0.5 * DHAT]])
    surf = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    sc, x = _scene(pts, surf, [[0, 1, 2]])
    lit = oracle.pairs(sc, x)
    dd = oracle.dedup(sc, x, lit)
    assert len(lit["type"]) == 1 and len(dd["type"]) == 1
    # two vertices over the same face are two feature pairs: both kept
    pts = np.array([[0.3, 0.3, 0.5 * DHAT], [0.2, 0.5, 0.7 * DHAT]])
    sc, x = _scene(pts, surf, [[0, 1, 2]])
    lit = oracle.pairs(sc, x)
    dd = oracle.dedup(sc, x, lit)
    assert len(lit["type"]) == 2 and len(dd["type"]) == 2


def _feature(sc, x, t, i, j, edge_of):
    if t == 0:
        v = [i, *sc.tris[j]]
    else:
        v = [*sc.edges[i], *sc.edges[j]]
    _, reg, _ = oracle.pair_d2(t, x[v].ravel())
    if t == 0:
        if reg == 0:
            return (0, j, i)
        if reg <= 3:
            e = reg - 1
            return (1, i, edge_of[tuple(sorted((v[1 + e], v[1 + (e + 1) % 3])))])
        return (2, *sorted((v[0], v[1 + reg - 4])))
    if reg == 0:
        return (3, i, j)
    if reg <= 4:
        e = reg - 1
        return (1, v[e], j if e < 2 else i)
    ia, ib = divmod(reg - 5, 2)
    return (2, *sorted((v[ia], v[2 + ib])))


@pytest.mark.parametrize("k", [1, 2])
def test_dedup_invariants_on_scenes(k):
    sc = scenes.make_config(k, small=(k == 2))
    x = oracle.embed(sc, sc.iterate(0))
    lit = oracle.pairs(sc, x)
    dd = oracle.dedup(sc, x, lit)
    edge_of = {tuple(e): n for n, e in enumerate(sc.edges.tolist())}
    kept = [(int(t), int(i), int(j)) for t, i, j in zip(dd["type"], dd["i"], dd["j"])]
    allp = [(int(t), int(i), int(j)) for t, i, j in zip(lit["type"], lit["i"], lit["j"])]
    assert kept == sorted(kept) and set(kept) <= set(allp)
    fk = [_feature(sc, x, *p, edge_of) for p in kept]
    assert len(set(fk)) == len(fk), "two kept pairs realise the same feature pair"
    fset = set(fk)
    dropped = set(allp) - set(kept)
    assert dropped, "no duplicates in this scene"
    for p in dropped:
        assert _feature(sc, x, *p, edge_of) in fset
    # a dropped pair comes after the kept pair of its feature in (type, i, j) order
    first = {}
    for p in allp:
        first.setdefault(_feature(sc, x, *p, edge_of), p)
    assert sorted(first.values()) == kept
    e_lit = oracle.eval_contact(sc, x, lit, None)["E"]
    e_dd = oracle.eval_contact(sc, x, dd, None)["E"]
    assert 0 < e_dd < e_lit
