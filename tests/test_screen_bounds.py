"""The lower bound behind the FP32 screen of near-parallel edge pairs (CPU only).

For segments A = a0 + s ea and B = b0 + t eb, the squared distance from the point of A at
parameter s to the line of B is |U + s V|^2 / |eb|^2 with U = (a0 - b0) x eb and
V = ea x eb.  Its minimum over s in [0, 1] is |U|^2 (U.V >= 0), |U + V|^2 (U.V <= -|V|^2),
else |U x V|^2 / |V|^2 (Lagrange's identity).  The segments' distance is at least that, and
at least the same bound with the roles swapped.  Checked here in FP64 against the oracle's
exact segment-segment distance, on near-parallel pairs of the sizes the contact stage sees.
"""
import numpy as np
import pytest

import oracle


def seg_line_min(U, V):
    uv, vv = U @ V, V @ V
    if uv >= 0.0:
        return U @ U
    if uv <= -vv:
        W = U + V
        return W @ W
    X = np.cross(U, V)
    return (X @ X) / vv


def seg_line_bound(a0, a1, b0, b1):
    ea, eb = a1 - a0, b1 - b0
    n = np.cross(ea, eb)
    lb_a = seg_line_min(np.cross(a0 - b0, eb), n) / (eb @ eb)
    lb_b = seg_line_min(np.cross(b0 - a0, ea), -n) / (ea @ ea)
    return max(lb_a, lb_b)


def _pair(rng, angle_max):
    a0 = rng.normal(size=3) * 1e-3
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    perp = np.cross(d, rng.normal(size=3))
    perp /= np.linalg.norm(perp)
    th = rng.uniform(0.0, angle_max)
    d2 = np.cos(th) * d + np.sin(th) * perp
    ea = d * rng.uniform(0.5e-3, 2e-3)
    eb = d2 * rng.uniform(0.5e-3, 2e-3) * rng.choice([1.0, -1.0])
    b0 = a0 + rng.normal(size=3) * rng.choice([2e-4, 1e-3, 3e-3])
    return a0, a0 + ea, b0, b0 + eb


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bound_never_exceeds_the_segment_distance(seed):
    rng = np.random.default_rng(seed)
    for _ in range(3000):
        a0, a1, b0, b1 = _pair(rng, 0.32)        # up to about 18 degrees
        lb = seg_line_bound(a0, a1, b0, b1)
        d2, _, _ = oracle.pair_d2(1, np.array([a0, a1, b0, b1]))
        assert lb <= d2 * (1.0 + 1e-9) + 1e-30, (lb, d2)


def test_bound_is_the_gap_of_parallel_surfaces():
    """Segments in two parallel planes a distance h apart: the bound is at least h^2, so a
    pair across a gap wider than dhat is proven far whatever its angle."""
    rng = np.random.default_rng(7)
    h = 2e-3
    for _ in range(500):
        a0 = np.array([*rng.normal(size=2) * 1e-3, 0.0])
        b0 = np.array([*rng.normal(size=2) * 1e-3, h])
        ea = np.array([*rng.normal(size=2), 0.0]) * 1e-3
        eb = np.array([*rng.normal(size=2), 0.0]) * 1e-3
        assert seg_line_bound(a0, a0 + ea, b0, b0 + eb) >= h * h * (1.0 - 1e-12)


def test_bound_is_exact_for_overlapping_parallel_segments():
    """Parallel segments that overlap along their common direction are the lateral offset
    apart, and the bound equals that distance squared."""
    a0, a1 = np.zeros(3), np.array([1e-3, 0.0, 0.0])
    b0, b1 = np.array([2e-4, 3e-4, 0.0]), np.array([8e-4, 3e-4, 0.0])
    assert abs(seg_line_bound(a0, a1, b0, b1) - 9e-8) <= 1e-20
