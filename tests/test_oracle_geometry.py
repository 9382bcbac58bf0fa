"""Pins for the oracle's unsigned distances (Sec. III-B, d_k of PT and EE pairs).

The distance of a pair is the minimum over the closed primitives; these tests pin the
oracle's closed-form minimisation against brute-force sampling of that minimum, against
closed forms of special configurations, and against the stencil it reports."""
import numpy as np
import pytest

import oracle

rng = np.random.default_rng(1234)


def _tri_samples(t0, t1, t2, n=120):
    u, v = np.meshgrid(np.linspace(0, 1, n + 1), np.linspace(0, 1, n + 1), indexing="ij")
    m = (u + v) <= 1.0 + 1e-15
    u = u[m]; v = v[m]
    return t0[None] + u[:, None] * (t1 - t0)[None] + v[:, None] * (t2 - t0)[None]


def _seg_samples(a, b, n=400):
    t = np.linspace(0, 1, n + 1)
    return a[None] + t[:, None] * (b - a)[None]


@pytest.mark.parametrize("trial", range(40))
def test_pt_distance_vs_sampling(trial):
    t = rng.normal(size=(3, 3))
    # mix of points over the face, near edges and past vertices
    p = t.mean(0) + rng.normal(size=3) * (0.3 + 1.5 * (trial % 3))
    d2, reg, c = oracle.pair_d2(0, np.concatenate([p, t.ravel()]))
    d = np.sqrt(d2)
    S = _tri_samples(*t)
    ds = np.sqrt(((S - p) ** 2).sum(1)).min()
    diam = max(np.linalg.norm(t[0] - t[1]), np.linalg.norm(t[1] - t[2]), np.linalg.norm(t[2] - t[0]))
    h = 1.0 / 120
    assert d <= ds + 1e-12
    assert ds <= d + h * diam
    # stencil: r = sum c_a x_a has length d
    X = np.vstack([p, t])
    r = (c[:, None] * X).sum(0)
    assert np.isclose(np.linalg.norm(r), d, rtol=1e-12, atol=1e-15)
    assert abs(c.sum()) < 1e-12


@pytest.mark.parametrize("trial", range(40))
def test_ee_distance_vs_sampling(trial):
    a0, a1, b0, b1 = rng.normal(size=(4, 3))
    if trial % 4 == 0:      # near-parallel
        b1 = b0 + (a1 - a0) * 0.8 + rng.normal(size=3) * 1e-4
    if trial % 8 == 1:      # exactly parallel
        b1 = b0 + 2.0 * (a1 - a0)
    d2, reg, c = oracle.pair_d2(1, np.concatenate([a0, a1, b0, b1]))
    d = np.sqrt(d2)
    A = _seg_samples(a0, a1); B = _seg_samples(b0, b1)
    ds = np.sqrt(((A[:, None] - B[None]) ** 2).sum(2)).min()
    la = np.linalg.norm(a1 - a0); lb = np.linalg.norm(b1 - b0)
    assert d <= ds + 1e-12
    assert ds <= d + (la + lb) / 400
    X = np.vstack([a0, a1, b0, b1])
    r = (c[:, None] * X).sum(0)
    assert np.isclose(np.linalg.norm(r), d, rtol=1e-10, atol=1e-14)
    assert abs(c.sum()) < 1e-12


def test_pt_closed_forms():
    t0 = np.array([0.0, 0.0, 0.0]); t1 = np.array([1.0, 0.0, 0.0]); t2 = np.array([0.0, 1.0, 0.0])
    # above the face interior: plane distance
    p = np.array([0.2, 0.3, 0.7])
    d2, reg, c = oracle.pair_d2(0, np.concatenate([p, t0, t1, t2]))
    assert reg == 0 and np.isclose(d2, 0.49, rtol=1e-15)
    assert np.allclose(c, [1, -0.5, -0.2, -0.3], atol=1e-15)
    # tilted triangle: n.(p - t0) / |n|
    T = rng.normal(size=(3, 3))
    n = np.cross(T[1] - T[0], T[2] - T[0]); n /= np.linalg.norm(n)
    p = T.mean(0) + 0.05 * n
    d2, reg, _ = oracle.pair_d2(0, np.concatenate([p, T.ravel()]))
    assert reg == 0 and np.isclose(np.sqrt(d2), 0.05, rtol=1e-12)
    # past vertex t1: point-point distance
    p = np.array([2.0, -1.0, 0.5])
    d2, reg, c = oracle.pair_d2(0, np.concatenate([p, t0, t1, t2]))
    assert reg == 5 and np.isclose(d2, 1 + 1 + 0.25)
    assert np.allclose(c, [1, 0, -1, 0])
    # beside edge t0-t1: distance to the line
    p = np.array([0.4, -0.3, 0.4])
    d2, reg, c = oracle.pair_d2(0, np.concatenate([p, t0, t1, t2]))
    assert reg == 1 and np.isclose(d2, 0.09 + 0.16)


def test_ee_closed_forms():
    # perpendicular crossing segments separated by 0.3 along z
    a0, a1 = np.array([-1.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0])
    b0, b1 = np.array([0.25, -1.0, 0.3]), np.array([0.25, 1.0, 0.3])
    d2, reg, c = oracle.pair_d2(1, np.concatenate([a0, a1, b0, b1]))
    assert reg == 0 and np.isclose(d2, 0.09, rtol=1e-15)
    assert np.allclose(c, [0.375, 0.625, -0.5, -0.5])
    # parallel overlapping segments: the distance between the lines
    b0, b1 = np.array([0.5, 0.2, 0.0]), np.array([3.0, 0.2, 0.0])
    d2, reg, _ = oracle.pair_d2(1, np.concatenate([a0, a1, b0, b1]))
    assert np.isclose(d2, 0.04, rtol=1e-14)
    # collinear disjoint: endpoint-endpoint
    b0, b1 = np.array([1.5, 0.0, 0.0]), np.array([3.0, 0.0, 0.0])
    d2, reg, c = oracle.pair_d2(1, np.concatenate([a0, a1, b0, b1]))
    assert np.isclose(d2, 0.25) and reg == 7


def test_ee_near_parallel_interior_minimum():
    """Segments crossing (in projection) at a small angle theta, one plane h above the
    other: the common perpendicular of the lines joins both midpoints, so d^2 = h^2 with
    the closest points inside both segments, while every endpoint is at least sin(theta)
    away.  Down to theta = 1e-4 (|ea x eb|^2 / (|ea|^2 |eb|^2) = 1e-8) the pair is not
    parallel and must take the interior minimum."""
    h = 0.01
    a0, a1 = np.array([-1.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0])
    for theta in (np.radians(5.0), np.radians(2.0), 1e-2, 1e-4):
        u = np.array([np.cos(theta), np.sin(theta), 0.0])
        b0, b1 = np.array([0.0, 0.0, h]) - u, np.array([0.0, 0.0, h]) + u
        d2, reg, c = oracle.pair_d2(1, np.concatenate([a0, a1, b0, b1]))
        assert reg == 0 and np.isclose(d2, h * h, rtol=1e-10), (theta, d2)
        assert np.allclose(c, [0.5, 0.5, -0.5, -0.5], atol=1e-8)


def test_degenerate_primitives():
    """A triangle with collinear vertices is the segment they span, and a zero-length edge is
    its point: the distances reduce to point-segment and point-point closed forms."""
    # collinear triangle on the x axis from 0 to 2 (vertex t2 in the middle)
    t0, t1, t2 = np.array([0.0, 0.0, 0.0]), np.array([2.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0])
    for p, expect in [((0.5, 0.3, 0.4), 0.25), ((-1.0, 0.0, 1.0), 2.0), ((1.5, -0.2, 0.0), 0.04)]:
        d2, reg, c = oracle.pair_d2(0, np.concatenate([p, t0, t1, t2]))
        assert np.isfinite(d2) and np.isclose(d2, expect, rtol=1e-14), (p, d2)
        assert reg != 0 and np.all(np.isfinite(c)) and abs(c.sum()) < 1e-14
    # random exactly collinear triangles (the 2x2 solve is singular, its determinant only
    # rounding): the distance to the segment they span
    r = np.random.default_rng(8)
    for _ in range(500):
        xs = r.uniform(-1e-3, 1e-3, 3)
        T = np.zeros((3, 3)); T[:, 0] = xs
        p = r.normal(size=3) * 1e-3
        d2, _, c = oracle.pair_d2(0, np.concatenate([p, T.ravel()]))
        t = np.clip(p[0], xs.min(), xs.max())
        assert np.isclose(d2, (p[0] - t) ** 2 + p[1] ** 2 + p[2] ** 2, rtol=1e-12)
        # the stencil weights still name the closest point
        assert np.isclose(np.linalg.norm(c[0] * p + c[1:] @ T), np.sqrt(d2), rtol=1e-9)
    # a triangle collapsed to one point
    P = np.array([0.3, -0.2, 0.1])
    d2, reg, _ = oracle.pair_d2(0, np.concatenate([[1.0, 1.0, 1.0], P, P, P]))
    assert np.isclose(d2, np.sum((np.array([1.0, 1.0, 1.0]) - P) ** 2), rtol=1e-14) and reg >= 4
    # edge-edge with one edge of zero length: point-segment distance
    a0 = a1 = np.array([0.5, 0.7, 0.2])
    b0, b1 = np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0])
    d2, reg, c = oracle.pair_d2(1, np.concatenate([a0, a1, b0, b1]))
    assert np.isclose(d2, 0.49 + 0.04, rtol=1e-14) and np.all(np.isfinite(c))


def test_distance_invariant_under_rigid_motion():
    for ptype in (0, 1):
        X = rng.normal(size=(4, 3))
        d2, _, _ = oracle.pair_d2(ptype, X.ravel())
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        Y = X @ Q.T + rng.normal(size=3)
        e2, _, _ = oracle.pair_d2(ptype, Y.ravel())
        assert np.isclose(d2, e2, rtol=1e-12)


def _two_tri_scene(V):
    from paper_2409_16385_gb300 import scenes
    tris = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    return scenes.Scene(name="pair", tris=tris, edges=scenes.edges_of(tris),
                        cage_idx=np.full((6, 4), -1, np.int32), w=np.zeros((6, 4)), x_kin=V, Ns=0,
                        cage_tets=np.zeros((0, 4), np.int32), q_rest=np.zeros((0, 3)),
                        body=np.zeros(6, np.int32), params={})


def test_intersection_test_on_exact_configurations():
    """The exact edge-triangle test behind the no-penetration checks (orientation
    predicates by expansion arithmetic): configurations decided by their exact geometry,
    including ones that floating-point rounding of a naive test would get wrong."""
    T = [[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]
    cases = [
        # an edge of the second triangle pierces the first one's interior
        ([[0.2, 0.2, -0.5], [0.3, 0.2, 0.5], [2.0, 2.0, 2.0]], False),
        # the same triangle lifted just above the plane: no contact
        ([[0.2, 0.2, 2.0 ** -50], [0.3, 0.2, 0.5], [2.0, 2.0, 2.0]], True),
        # a vertex exactly on the first triangle's interior: the closed sets meet
        ([[0.25, 0.25, 0.0], [0.3, 0.2, 0.5], [2.0, 2.0, 2.0]], False),
        # coplanar and overlapping
        ([[0.1, 0.1, 0.0], [2.0, 0.1, 0.0], [0.1, 2.0, 0.0]], False),
        # coplanar and disjoint (beyond the hypotenuse x + y = 1)
        ([[0.6, 0.6, 0.0], [2.0, 0.6, 0.0], [0.6, 2.0, 0.0]], True),
        # an edge passing exactly through the hypotenuse's midpoint, off the plane elsewhere
        ([[0.5, 0.5, -1.0], [0.5, 0.5, 1.0], [3.0, 3.0, 0.5]], False),
        # the same edge shifted by the smallest step beyond the hypotenuse
        ([[0.5, np.nextafter(0.5, 1.0), -1.0], [0.5, np.nextafter(0.5, 1.0), 1.0], [3.0, 3.0, 0.5]], True),
    ]
    for upper, free in cases:
        V = np.array(T + upper, float)
        assert oracle.intersection_free(_two_tri_scene(V), V) is free, (upper, free)
    # large integer coordinates: the plane x + y + z = 2^30 holds the first triangle, and a
    # vertex with coordinate sum exactly 2^30 lies on it.  The orientation determinants
    # reach 2^90, far beyond what one FP64 rounding can decide.
    G = 2.0 ** 30
    T = [[G, 0.0, 0.0], [0.0, G, 0.0], [0.0, 0.0, G]]
    on = [2.0 ** 29 + 3, 2.0 ** 29 - 5, 2.0]
    for lift, free in ((0.0, False), (1.0, True), (-1.0, False)):
        up = [[on[0], on[1], on[2] + lift], [G, G, G], [G, 2 * G, G]]
        V = np.array(T + up, float)
        assert oracle.intersection_free(_two_tri_scene(V), V) is free, (lift, free)
