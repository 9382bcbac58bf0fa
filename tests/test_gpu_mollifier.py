"""GPU parity of the EE mollifier (eipc_scene_set_mollifier) on two nearly parallel sheets,
where about a fifth of the pairs are mollified: E, g_r, H_r (projected and exact), the
exact HVP and the lagged normal forces against the oracle with the same mollifier."""
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


@pytest.fixture
def sheets():
    sc = scenes.parallel_sheets()
    xr = oracle.embed(sc, sc.q_rest)
    oracle.set_mollifier(sc, xr)
    yield sc, xr
    oracle.set_mollifier(sc, None)


def _bsr(H, ns):
    h = H.host()
    return {(r, int(h["col"][k])): h["val"][k] for r in range(ns) for k in range(h["row_ptr"][r], h["row_ptr"][r + 1])}


@pytest.mark.parametrize("project", [True, False])
def test_mollified_evaluation_matches_oracle(sheets, project):
    from paper_2409_16385_gb300 import ContactScene
    sc, xr = sheets
    cs = ContactScene(sc, pair_capacity=1 << 18, bsr_capacity=1 << 19, rec_capacity=1 << 22)
    cs.set_mollifier(xr)
    q0, q1 = _t(sc.iterate(0)), _t(sc.iterate(1))
    lag = cs.friction_lag(q0, cs.build_candidates(q0, out=cs.new_pairs()))
    pairs = cs.build_candidates(q1)
    E, g, H = cs.eval_contact(q1, pairs, lag, project=project)
    torch.cuda.synchronize()
    assert cs.status()["flags"] == 0
    x0, x1 = oracle.embed(sc, sc.iterate(0)), oracle.embed(sc, sc.iterate(1))
    h = pairs.host()
    prs = dict(type=h["type"], i=h["i"], j=h["j"])
    lo = oracle.friction_lag(sc, x0, oracle.pairs(sc, x0))
    lg = lag.host()
    assert np.allclose(lg["lam"], lo["lam"], rtol=1e-9, atol=0)
    ro = oracle.eval_contact(sc, x1, prs, lo, project=project)
    assert abs(float(E.item()) - ro["E"]) <= TOL * abs(ro["E"])
    assert np.abs(g.cpu().numpy() - ro["g"]).max() <= TOL * np.abs(ro["g"]).max()
    hg = _bsr(H, sc.Ns)
    ho = {(int(a), int(b)): v for a, b, v in zip(ro["I"], ro["J"], ro["V"])}
    assert set(hg) == set(ho)
    hs = max(np.abs(v).max() for v in ho.values())
    assert max(np.abs(hg[k] - ho[k]).max() for k in ho) <= TOL * hs
    # the mollifier changes the result (it is on)
    cs.set_mollifier(None)
    E2, _, _ = cs.eval_contact(q1, pairs, lag, project=project)
    assert abs(float(E2.item()) - float(E.item())) > 1e-6 * abs(float(E.item()))


def test_mollified_hvp_matches_oracle(sheets):
    from paper_2409_16385_gb300 import ContactScene
    sc, xr = sheets
    cs = ContactScene(sc, pair_capacity=1 << 18, bsr_capacity=1 << 19, rec_capacity=1 << 22)
    cs.set_mollifier(xr)
    q0, q1 = _t(sc.iterate(0)), _t(sc.iterate(1))
    lag = cs.friction_lag(q0, cs.build_candidates(q0, out=cs.new_pairs()))
    pairs = cs.build_candidates(q1)
    v = np.random.default_rng(4).normal(size=(sc.Ns, 3))
    kd = np.array([0.1, -0.3, 1.0])
    out, out_kin = cs.contact_hvp(q1, pairs, _t(v), lag=lag, kin_dir=kd)
    torch.cuda.synchronize()
    x0, x1 = oracle.embed(sc, sc.iterate(0)), oracle.embed(sc, sc.iterate(1))
    h = pairs.host()
    prs = dict(type=h["type"], i=h["i"], j=h["j"])
    lo = oracle.friction_lag(sc, x0, oracle.pairs(sc, x0))
    u = oracle.embed(sc, v, displacement=True)
    u[sc.kinematic] = kd
    ro, rk = oracle.hvp(sc, x1, prs, lo, u)
    assert np.abs(out.cpu().numpy() - ro).max() <= TOL * np.abs(ro).max()
    assert np.abs(out_kin.cpu().numpy() - rk).max() <= TOL * np.abs(rk).max()


def test_mollifier_rest_lengths_are_checked_in_the_library():
    """The library takes the rest positions and computes the edges' squared rest lengths
    itself; a zero-length edge at rest is refused and leaves the mollifier off."""
    from paper_2409_16385_gb300 import ContactScene
    sc = scenes.parallel_sheets()
    xr = oracle.embed(sc, sc.q_rest)
    cs = ContactScene(sc, pair_capacity=1 << 18, bsr_capacity=1 << 19, rec_capacity=1 << 22)
    q1 = _t(sc.iterate(1))
    pairs = cs.build_candidates(q1)
    E_off, _, _ = cs.eval_contact(q1, pairs)
    bad = xr.copy()
    a, b = sc.edges[7]
    bad[b] = bad[a]
    with pytest.raises(RuntimeError):
        cs.set_mollifier(bad)
    E_bad, _, _ = cs.eval_contact(q1, pairs)
    assert E_bad.item() == E_off.item()
    cs.set_mollifier(xr)
    E_on, _, _ = cs.eval_contact(q1, pairs)
    assert E_on.item() != E_off.item()
