"""Pins for the oracle's barrier, friction mollifier, per-pair derivatives and PSD
projection (Sec. III-B Eq. 7, Eqs. 8-9; Sec. III-C projected Newton)."""
import json
import os

import numpy as np
import pytest

import oracle

rng = np.random.default_rng(99)
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _paper_params():
    with open(os.path.join(GOLD, "paper_parameters.json")) as f:
        return json.load(f)


# ----------------------------------------------------------------------- barrier b(d)

def test_barrier_closed_form_and_boundary():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    dhat = _paper_params()["bubble_gripper"]["dhat"]
    for d in [1e-9, 1e-6, 3e-4, 0.5e-3, 0.999e-3]:
        b, b1, b2 = oracle.barrier(d, dhat)
        D, H = mp.mpf(d), mp.mpf(dhat)
        f = lambda z: -(z - H) ** 2 * mp.log(z / H)
        assert np.isclose(b, float(f(D)), rtol=1e-13, atol=0)
        assert np.isclose(b1, float(mp.diff(f, D)), rtol=1e-10)
        assert np.isclose(b2, float(mp.diff(f, D, 2)), rtol=1e-8)
        assert b > 0
    # b(dhat) = b'(dhat) = 0 and b vanishes outside (0, dhat)
    assert np.all(oracle.barrier(dhat, dhat) == 0)
    assert np.all(oracle.barrier(2 * dhat, dhat) == 0)
    b_in = oracle.barrier(dhat * (1 - 1e-7), dhat)
    assert abs(b_in[0]) < 1e-18 and abs(b_in[1]) < 1e-12


# ----------------------------------------------------------------------- friction f0

def test_f0_matches_integral_of_f1():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    pp = _paper_params()["bubble_gripper"]
    eps = pp["eps_v"] * 0.01

    def f1(y):   # Eq. 9
        return -y * y / (eps * eps) + 2 * y / eps if y < eps else mp.mpf(1)

    for y in [0.0, 1e-8, 0.3 * eps, 0.9 * eps, eps, 1.7 * eps, 5 * eps]:
        ref = mp.quad(f1, [eps, y]) + eps if y != eps else mp.mpf(eps)
        f, fp, fpp = oracle.f0(y, eps)
        assert np.isclose(f, float(ref), rtol=1e-12, atol=1e-20)
        assert np.isclose(fp, float(f1(mp.mpf(y))), rtol=1e-12, atol=1e-14)
    # C1 across eps
    lo = oracle.f0(eps * (1 - 1e-9), eps); hi = oracle.f0(eps * (1 + 1e-9), eps)
    assert np.isclose(lo[0], hi[0], rtol=1e-8) and np.isclose(lo[1], hi[1], rtol=1e-6)
    assert np.isclose(oracle.f0(0.0, eps)[0], eps / 3)


# ----------------------------------------------------------------------- derivatives

def _random_pair(ptype, dhat, region):
    """A random stencil at distance ~0.5 dhat in a chosen region."""
    while True:
        T = rng.normal(size=(3, 3)) * 1e-2
        if ptype == 0:
            n = np.cross(T[1] - T[0], T[2] - T[0]); n /= np.linalg.norm(n)
            if region == "face":
                p = T.mean(0) + 0.5 * dhat * n
            elif region == "edge":
                m = 0.5 * (T[0] + T[1]); out = m - T[2]; out -= (out @ n) * n
                p = m + 0.3 * dhat * out / np.linalg.norm(out) + 0.4 * dhat * n
            else:
                out = T[0] - T.mean(0)
                p = T[0] + 0.5 * dhat * out / np.linalg.norm(out)
            x4 = np.concatenate([p, T.ravel()])
        else:
            a0, a1 = rng.normal(size=(2, 3)) * 1e-2
            u = rng.normal(size=3); u -= (u @ (a1 - a0)) / ((a1 - a0) @ (a1 - a0)) * (a1 - a0)
            mid = 0.5 * (a0 + a1)
            dirb = np.cross(a1 - a0, u); dirb /= np.linalg.norm(dirb)
            off = 0.5 * dhat * u / np.linalg.norm(u)
            if region == "face":   # interior-interior
                b0 = mid + off - 0.01 * dirb; b1 = mid + off + 0.01 * dirb
            elif region == "edge":  # endpoint of b against interior of a
                b0 = mid + off; b1 = mid + off + 0.01 * (dirb + u / np.linalg.norm(u))
            else:                   # endpoint-endpoint
                b0 = a1 + 0.5 * dhat * (a1 - a0) / np.linalg.norm(a1 - a0)
                b1 = b0 + 0.01 * rng.normal(size=3)
            x4 = np.concatenate([a0, a1, b0, b1])
        d2, reg, _ = oracle.pair_d2(ptype, x4)
        if 0 < np.sqrt(d2) < dhat:
            return x4, reg


@pytest.mark.parametrize("ptype", [0, 1])
@pytest.mark.parametrize("region", ["face", "edge", "vertex"])
def test_barrier_derivatives_vs_central_differences(ptype, region):
    dhat, kappa = 1e-3, 1e4
    for _ in range(3):
        x4, reg = _random_pair(ptype, dhat, region)
        E, g, H, _ = oracle.pair_barrier(ptype, x4, dhat, kappa)
        h = 1e-7 * 1e-2
        gfd = np.zeros(12); Hfd = np.zeros((12, 12))
        for i in range(12):
            e = np.zeros(12); e[i] = h
            Ep = oracle.pair_barrier(ptype, x4 + e, dhat, kappa)
            Em = oracle.pair_barrier(ptype, x4 - e, dhat, kappa)
            gfd[i] = (Ep[0] - Em[0]) / (2 * h)
            Hfd[:, i] = (Ep[1] - Em[1]) / (2 * h)
        assert np.abs(g - gfd).max() <= 1e-6 * np.abs(g).max()
        assert np.abs(H - Hfd).max() <= 1e-5 * np.abs(H).max()
        assert np.allclose(H, H.T, atol=1e-12 * np.abs(H).max())
        # translation invariance of the pair energy
        for k in range(3):
            assert abs(g[k::3].sum()) <= 1e-9 * np.abs(g).max()


def test_point_point_hessian_closed_form():
    # vertex region: d^2 = |p - t0|^2, so hess(kappa b(d)) has a closed form
    dhat, kappa = 1e-3, 1e4
    T = np.array([[0.0, 0, 0], [0.01, 0, 0], [0, 0.01, 0]])
    dirn = np.array([-1.0, -2.0, 0.5]); dirn /= np.linalg.norm(dirn)
    d = 0.4 * dhat
    p = T[0] + d * dirn
    E, g, H, Hp = oracle.pair_barrier(0, np.concatenate([p, T.ravel()]), dhat, kappa)
    b, b1, b2 = oracle.barrier(d, dhat)
    assert np.isclose(E, kappa * b)
    A = kappa * (b2 * np.outer(dirn, dirn) + (b1 / d) * (np.eye(3) - np.outer(dirn, dirn)))
    Hc = np.zeros((12, 12))
    Hc[0:3, 0:3] = A; Hc[3:6, 3:6] = A; Hc[0:3, 3:6] = -A; Hc[3:6, 0:3] = -A
    assert np.allclose(H, Hc, rtol=1e-10, atol=1e-10 * np.abs(Hc).max())
    # projected: only the radial stiffness survives (b'' > 0, b'/d < 0)
    Ap = kappa * b2 * np.outer(dirn, dirn)
    Hpc = np.zeros((12, 12))
    Hpc[0:3, 0:3] = Ap; Hpc[3:6, 3:6] = Ap; Hpc[0:3, 3:6] = -Ap; Hpc[3:6, 0:3] = -Ap
    assert np.allclose(Hp, Hpc, atol=1e-9 * np.abs(Hpc).max())


# ----------------------------------------------------------------------- PSD projection

def test_psd_projection_properties():
    for n in (3, 6, 12):
        for _ in range(5):
            A = rng.normal(size=(n, n)); H = A + A.T
            lam, V = oracle.eigen(H)
            assert np.allclose(np.sort(lam), np.linalg.eigvalsh(H), atol=1e-12 * np.abs(H).max())
            Hp = oracle.psd_project(H)
            # the textbook definition via a library eigensolver
            w, U = np.linalg.eigh(H)
            ref = (U * np.maximum(w, 0)) @ U.T
            assert np.allclose(Hp, ref, atol=1e-12 * np.abs(H).max())
            assert np.linalg.eigvalsh(Hp).min() >= -1e-12 * np.abs(H).max()
            assert np.allclose(oracle.psd_project(Hp), Hp, atol=1e-12 * np.abs(H).max())
            P = A @ A.T
            assert np.allclose(oracle.psd_project(P), P, atol=1e-12 * np.abs(P).max())


def test_projected_barrier_hessian_is_psd_and_nearest():
    dhat, kappa = 1e-3, 1e4
    for ptype in (0, 1):
        for region in ("face", "edge"):
            x4, _ = _random_pair(ptype, dhat, region)
            _, _, H, Hp = oracle.pair_barrier(ptype, x4, dhat, kappa)
            w, U = np.linalg.eigh(H)
            assert w.min() < 0      # the raw barrier Hessian is indefinite
            assert np.allclose(Hp, (U * np.maximum(w, 0)) @ U.T, atol=1e-11 * np.abs(H).max())


# ----------------------------------------------------------------------- friction

def test_friction_derivatives_and_invariants():
    mu, eps, lam = 0.5, 1e-5, 3.7
    for ptype in (0, 1):
        x4n, _ = _random_pair(ptype, 1e-3, "face")
        d2, reg, c = oracle.pair_d2(ptype, x4n)
        X = x4n.reshape(4, 3)
        r = (c[:, None] * X).sum(0)
        n = r / np.linalg.norm(r)
        anchor = r.copy()
        v4 = np.arange(4)
        # at x = x^n: u = 0 -> E = mu lam eps/3, zero gradient
        E, g, H = oracle.pair_friction(v4, c, n, anchor, lam, x4n, mu, eps)
        assert np.isclose(E, mu * lam * eps / 3) and np.abs(g).max() == 0
        for scale in (0.3 * eps, 4 * eps):   # both branches of f0
            t = rng.normal(size=3); t -= (t @ n) * n; t /= np.linalg.norm(t)
            x4 = x4n.copy(); x4[0:3] += scale * t / abs(c[0])
            E, g, H = oracle.pair_friction(v4, c, n, anchor, lam, x4, mu, eps)
            u = np.linalg.norm((c[:, None] * x4.reshape(4, 3)).sum(0) - anchor - 0 * n)
            assert np.isclose(E, mu * lam * oracle.f0(u, eps)[0], rtol=1e-12)
            h = 1e-3 * eps
            gfd = np.zeros(12); Hfd = np.zeros((12, 12))
            for i in range(12):
                e = np.zeros(12); e[i] = h
                Ep = oracle.pair_friction(v4, c, n, anchor, lam, x4 + e, mu, eps)
                Em = oracle.pair_friction(v4, c, n, anchor, lam, x4 - e, mu, eps)
                gfd[i] = (Ep[0] - Em[0]) / (2 * h)
                Hfd[:, i] = (Ep[1] - Em[1]) / (2 * h)
            assert np.abs(g - gfd).max() <= 1e-6 * np.abs(g).max()
            assert np.abs(H - Hfd).max() <= 1e-5 * np.abs(H).max()
            assert np.linalg.eigvalsh(H).min() >= -1e-10 * np.abs(H).max()   # already PSD
            # motion along the normal is not friction
            x4b = x4.copy(); x4b[0:3] += 1e-4 * n / c[0]
            Eb, _, _ = oracle.pair_friction(v4, c, n, anchor, lam, x4b, mu, eps)
            assert np.isclose(Eb, E, rtol=1e-12)


def test_friction_hessian_at_zero_slip_is_the_limit():
    """At x = x^n the tangential slip u is 0 and the oracle takes the Hessian's limit
    (Sec. III-B with Eq. 9: f1(y) / y -> 2 / eps).  Pinned against central differences of
    the gradient around x^n, which the general branch computes (u != 0 on both sides)."""
    mu, eps, lam = 0.5, 1e-5, 3.7
    for ptype in (0, 1):
        x4n, _ = _random_pair(ptype, 1e-3, "face")
        d2, reg, c = oracle.pair_d2(ptype, x4n)
        X = x4n.reshape(4, 3)
        r = (c[:, None] * X).sum(0)
        n = r / np.linalg.norm(r)
        v4 = np.arange(4)
        E, g, H = oracle.pair_friction(v4, c, n, r, lam, x4n, mu, eps)
        assert np.abs(g).max() == 0
        h = 1e-6 * eps
        Hfd = np.zeros((12, 12))
        for i in range(12):
            e = np.zeros(12); e[i] = h
            gp = oracle.pair_friction(v4, c, n, r, lam, x4n + e, mu, eps)[1]
            gm = oracle.pair_friction(v4, c, n, r, lam, x4n - e, mu, eps)[1]
            Hfd[:, i] = (gp - gm) / (2 * h)
        assert np.abs(H).max() > 0
        assert np.abs(H - Hfd).max() <= 1e-5 * np.abs(H).max()
