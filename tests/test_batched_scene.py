"""The batched-scene generator: a batch is its scenes side by side, and the oracle sees
no interaction between them (CPU only)."""
import numpy as np

import oracle
from paper_2409_16385_gb300 import scenes


def _tiny_batch():
    return scenes.batched_grasp(n_scenes=4, seed=3, min_tris=300, max_tris=900)


def test_parts_are_contiguous_slices_of_the_batch():
    b = scenes.make_config(4, small=True)
    assert b.n_scenes == 16
    for s in range(b.n_scenes):
        p = b.part_scene(s)
        v0, nv = b.vertex_ranges[s]
        f0, nf = b.tri_ranges[s]
        e0, ne = b.edge_ranges[s]
        n0, ns = b.node_ranges[s]
        assert np.array_equal(b.tris[f0:f0 + nf] - v0, p.tris)
        assert np.array_equal(b.edges[e0:e0 + ne] - v0, p.edges)
        ci = b.cage_idx[v0:v0 + nv].copy()
        ci[ci >= 0] -= n0
        assert np.array_equal(ci, p.cage_idx)
        assert np.array_equal(b.w[v0:v0 + nv], p.w)
        assert np.array_equal(b.x_kin[v0:v0 + nv], p.x_kin)
        assert np.all(b.body[v0:v0 + nv] == s)
        for t in (0, 11, b.n_iterates - 1):
            assert np.array_equal(b.iterate(t)[n0:n0 + ns], p.iterate(t))
            assert np.array_equal(b.dq(t)[n0:n0 + ns], p.dq(t))
    # sizes are uneven and phases differ
    sizes = [sc.F for sc, _ in b.parts]
    assert max(sizes) > 2 * min(sizes)
    assert len({ph for _, ph in b.parts}) > 4
    assert all(ph % 3 == 0 for _, ph in b.parts)


def test_oracle_batch_is_the_sum_of_its_scenes():
    """Contact set, energy, reduced gradient and step bound of the batch are those of its
    scenes evaluated one by one: the grid spacing keeps scenes apart."""
    b = _tiny_batch()
    t = 5
    x = oracle.embed(b, b.iterate(t))
    po = oracle.pairs(b, x)
    ro = oracle.eval_contact(b, x, po, None)
    alpha = oracle.accd(b, x, oracle.embed(b, b.dq(t), displacement=True))["alpha"]
    E, n, amin = 0.0, 0, 1.0
    for s in range(b.n_scenes):
        p = b.part_scene(s)
        xs = oracle.embed(p, p.iterate(t))
        ps = oracle.pairs(p, xs)
        rs = oracle.eval_contact(p, xs, ps, None)
        n0, ns = b.node_ranges[s]
        assert np.allclose(ro["g"][n0:n0 + ns], rs["g"], rtol=0, atol=1e-12 * max(1.0, np.abs(rs["g"]).max()))
        E += rs["E"]
        n += len(ps["type"])
        amin = min(amin, oracle.accd(p, xs, oracle.embed(p, p.dq(t), displacement=True))["alpha"])
    assert n == len(po["type"]) and n > 0
    assert abs(E - ro["E"]) <= 1e-12 * abs(ro["E"])
    assert alpha == amin
