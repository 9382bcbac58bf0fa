"""Pins of the oracle's EE mollifier (CPU only).

The mollified pair energy kappa m(c) b(d) against its closed form (c = |e0 x e1|^2 from
numpy, d from the oracle's distance, b and m written out), its gradient and Hessian
against central differences, no change above eps_x, continuity across c = eps_x, and on
a scene of nearly parallel sheets: a lower energy with the mollifier, unchanged above the
threshold, and lagged normal forces scaled by m.
"""
import numpy as np

import oracle
from paper_2409_16385_gb300 import scenes

DHAT, KAPPA = 1e-3, 1e4


def _b(d):
    return -(d - DHAT) ** 2 * np.log(d / DHAT)


def _m(c, eps):
    return c * (2.0 / eps - c / eps ** 2) if c < eps else 1.0


def _edges(angle, gap=0.4e-3, shift=0.0):
    a0, a1 = np.array([-1e-3, 0, 0]), np.array([1e-3, 0, 0])
    dirb = np.array([np.cos(angle), np.sin(angle), 0.0])
    b0 = np.array([shift, 0, gap]) - 1.2e-3 * dirb
    b1 = np.array([shift, 0, gap]) + 1.2e-3 * dirb
    return np.concatenate([a0, a1, b0, b1])


def _c(x4):
    x = x4.reshape(4, 3)
    n = np.cross(x[1] - x[0], x[3] - x[2])
    return float(n @ n)


def test_energy_matches_the_closed_form():
    for angle in (1e-3, 5e-3, 0.02):
        x4 = _edges(angle)
        eps = 1e-3 * (2e-3) ** 2 * (2.4e-3) ** 2
        E, _, _ = oracle.pair_barrier_mollified(x4, eps, DHAT, KAPPA)
        d = np.sqrt(oracle.pair_d2(1, x4)[0])
        ref = KAPPA * _m(_c(x4), eps) * _b(d)
        assert abs(E - ref) <= 1e-13 * abs(ref)


def test_derivatives_match_central_differences():
    rng = np.random.default_rng(0)
    x4 = _edges(4e-3) + 1e-5 * rng.normal(size=12)
    eps = 1e-3 * (2e-3) ** 2 * (2.4e-3) ** 2
    assert _c(x4) < eps
    E, g, H = oracle.pair_barrier_mollified(x4, eps, DHAT, KAPPA)
    for _ in range(3):
        v = rng.normal(size=12)
        h = 1e-9
        fe = (oracle.pair_barrier_mollified(x4 + h * v, eps, DHAT, KAPPA)[0]
              - oracle.pair_barrier_mollified(x4 - h * v, eps, DHAT, KAPPA)[0]) / (2 * h)
        assert abs(fe - g @ v) <= 1e-6 * np.abs(g).max() * np.abs(v).max()
        fg = (oracle.pair_barrier_mollified(x4 + h * v, eps, DHAT, KAPPA)[1]
              - oracle.pair_barrier_mollified(x4 - h * v, eps, DHAT, KAPPA)[1]) / (2 * h)
        assert np.abs(fg - H @ v).max() <= 1e-6 * np.abs(H @ v).max()
    assert np.allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())


def test_no_change_above_the_threshold_and_continuity_at_it():
    x4 = _edges(0.3)
    eps = 1e-12
    E, g, H = oracle.pair_barrier_mollified(x4, eps, DHAT, KAPPA)
    E0, g0, H0, _ = oracle.pair_barrier(1, x4, DHAT, KAPPA)
    assert E == E0 and np.array_equal(g, g0) and np.array_equal(H, H0)
    # also where c is only a little above eps_x: m = 1 for every c >= eps_x
    x4 = _edges(4e-3)
    E, g, H = oracle.pair_barrier_mollified(x4, _c(x4) / 1.5, DHAT, KAPPA)
    E0, g0, H0, _ = oracle.pair_barrier(1, x4, DHAT, KAPPA)
    assert E == E0 and np.array_equal(g, g0) and np.array_equal(H, H0)
    c = _c(x4)
    lo = oracle.pair_barrier_mollified(x4, c * (1 - 1e-9), DHAT, KAPPA)
    hi = oracle.pair_barrier_mollified(x4, c * (1 + 1e-9), DHAT, KAPPA)
    assert abs(lo[0] - hi[0]) <= 1e-8 * abs(lo[0])
    assert np.abs(lo[1] - hi[1]).max() <= 1e-6 * np.abs(lo[1]).max()


def test_scene_energy_and_lag_with_the_mollifier():
    sc = scenes.parallel_sheets()
    x = oracle.embed(sc, sc.iterate(0))
    prs = oracle.pairs(sc, x)
    xr = oracle.embed(sc, sc.q_rest)
    try:
        e_plain = oracle.eval_contact(sc, x, prs, None)["E"]
        lag_plain = oracle.friction_lag(sc, x, prs)
        oracle.set_mollifier(sc, xr)
        e_moll = oracle.eval_contact(sc, x, prs, None)["E"]
        lag_moll = oracle.friction_lag(sc, x, prs)
    finally:
        oracle.set_mollifier(sc, None)
    assert 0 < e_moll < e_plain
    e = sc.edges
    r2 = np.sum((xr[e[:, 1]] - xr[e[:, 0]]) ** 2, axis=1)
    ee = prs["type"] == 1
    i, j = prs["i"][ee], prs["j"][ee]
    cc = np.sum(np.cross(x[e[i, 1]] - x[e[i, 0]], x[e[j, 1]] - x[e[j, 0]]) ** 2, axis=1)
    eps = 1e-3 * r2[i] * r2[j]
    m = np.where(cc < eps, cc * (2 / eps - cc / eps ** 2), 1.0)
    assert (cc < eps).sum() > 100
    assert np.allclose(lag_moll["lam"][ee], m * lag_plain["lam"][ee], rtol=1e-12, atol=0)
    assert np.array_equal(lag_moll["lam"][~ee], lag_plain["lam"][~ee])
