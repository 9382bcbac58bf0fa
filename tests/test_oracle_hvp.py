"""Pins of the oracle's Hessian-vector product of the contact potential (CPU only).

oracle.hvp applies the unprojected contact Hessian (barrier and lagged friction) to a
full-space direction.  It is pinned to
  * central differences of the oracle's reduced gradient g_r along a reduced direction v
    (the pair list and the friction lag held fixed, so g_r is a smooth function of q),
  * central differences of g_r under a rigid shift of the kinematic vertices,
  * symmetry of the full Hessian: <v, d g_r/d shift . e> = <e, sum_kin (H J v)>,
  * the unprojected reduced Hessian that orc_eval assembles block by block.
"""
import dataclasses
import functools

import numpy as np

import oracle
from paper_2409_16385_gb300 import scenes


@functools.lru_cache(maxsize=None)
def _setup():
    sc = scenes.make_config(1)
    q0 = sc.iterate(0)
    x0 = oracle.embed(sc, q0)
    p0 = oracle.pairs(sc, x0)
    lag = oracle.friction_lag(sc, x0, p0)
    a = oracle.accd(sc, x0, oracle.embed(sc, sc.dq(0), displacement=True))["alpha"]
    sc2 = scenes.with_second_iterate(sc, a)
    q1 = sc2.iterate(1)
    x1 = oracle.embed(sc2, q1)
    p1 = oracle.pairs(sc2, x1)
    return sc2, q1, p1, lag


def _g(sc, q, prs, lag):
    return oracle.eval_contact(sc, oracle.embed(sc, q), prs, lag)["g"]


def _dir(sc, seed):
    v = np.random.default_rng(seed).normal(size=(sc.Ns, 3))
    return v / np.abs(v).max() * 1e-3


def test_hvp_matches_central_differences_of_the_gradient():
    sc, q, prs, lag = _setup()
    assert len(prs["type"]) > 50 and len(lag["lam"]) > 20
    v = _dir(sc, 1)
    u = oracle.embed(sc, v, displacement=True)
    hv, _ = oracle.hvp(sc, oracle.embed(sc, q), prs, lag, u)
    # d^2 is only C^1 across closest-feature regions and one pair of this configuration lies
    # within 1e-7 m of a region boundary, so the step moves vertices by at most 1e-8 m
    eps = 1e-5
    fd = (_g(sc, q + eps * v, prs, lag) - _g(sc, q - eps * v, prs, lag)) / (2 * eps)
    assert np.abs(hv).max() > 0
    assert np.abs(fd - hv).max() <= 1e-7 * np.abs(hv).max()


def test_hvp_of_a_kinematic_shift_matches_central_differences():
    sc, q, prs, lag = _setup()
    kin = sc.kinematic
    x = oracle.embed(sc, q)
    for axis in range(3):
        e = np.zeros(3); e[axis] = 1.0
        u = np.zeros((sc.Nv, 3)); u[kin] = e
        hv, _ = oracle.hvp(sc, x, prs, lag, u)
        eps = 1e-9          # a pad vertex lies within 1e-8 m of a region boundary
        shifted = []
        for sgn in (1, -1):
            s2 = dataclasses.replace(sc, x_kin=np.where(kin[:, None], sc.x_kin + sgn * eps * e, sc.x_kin))
            shifted.append(_g(s2, q, prs, lag))
        fd = (shifted[0] - shifted[1]) / (2 * eps)
        scale = np.abs(hv).max()
        assert scale > 0
        assert np.abs(fd - hv).max() <= 1e-7 * scale, axis


def test_kinematic_sum_balances_the_reduced_rows():
    """The contact potential is invariant under a common translation of every vertex (on
    each side of a pair the closest-point weights sum to 1, resp. -1), so its Hessian
    times any u sums to zero over all vertices.  The embedding weights of a vertex sum to 1,
    so the reduced rows sum to the embedded vertices' part: the kinematic sum is minus the
    sum of the reduced rows."""
    sc, q, prs, lag = _setup()
    x = oracle.embed(sc, q)
    r = np.random.default_rng(3)
    for _ in range(3):
        u = r.normal(size=(sc.Nv, 3))
        hv, kin_sum = oracle.hvp(sc, x, prs, lag, u)
        scale = np.abs(hv).sum(0).max()
        assert np.abs(kin_sum).max() > 1e-3 * scale
        assert np.abs(kin_sum + hv.sum(0)).max() <= 1e-10 * scale


def test_mixed_blocks_are_symmetric():
    sc, q, prs, lag = _setup()
    kin = sc.kinematic
    x = oracle.embed(sc, q)
    v = _dir(sc, 2)
    _, kin_sum = oracle.hvp(sc, x, prs, lag, oracle.embed(sc, v, displacement=True))
    for axis in range(3):
        e = np.zeros(3); e[axis] = 1.0
        u = np.zeros((sc.Nv, 3)); u[kin] = e
        hv, _ = oracle.hvp(sc, x, prs, lag, u)
        a, b = float(np.sum(v * hv)), float(kin_sum[axis])
        assert abs(a - b) <= 1e-12 * max(abs(a), abs(b), 1e-300), (axis, a, b)


def test_hvp_equals_the_unprojected_reduced_hessian():
    sc, q, prs, lag = _setup()
    x = oracle.embed(sc, q)
    r = oracle.eval_contact(sc, x, prs, lag, project=False)
    v = _dir(sc, 3)
    hv, _ = oracle.hvp(sc, x, prs, lag, oracle.embed(sc, v, displacement=True))
    ref = np.zeros_like(v)
    for I, J, B in zip(r["I"], r["J"], r["V"]):
        ref[I] += B @ v[J]
    assert np.abs(ref - hv).max() <= 1e-12 * np.abs(ref).max()
    # the projected Hessian differs: some pair Hessians are indefinite here
    rp = oracle.eval_contact(sc, x, prs, lag, project=True)
    refp = np.zeros_like(v)
    for I, J, B in zip(rp["I"], rp["J"], rp["V"]):
        refp[I] += B @ v[J]
    assert np.abs(refp - hv).max() > 1e-9 * np.abs(ref).max()
