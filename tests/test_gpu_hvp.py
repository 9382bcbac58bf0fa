"""GPU parity of the exact (unprojected) contact Hessian: eipc_contact_hvp and
eipc_eval_contact with EIPC_PARAM_NO_PROJECTION, against the oracle (1e-9 relative), and
the kinematic-position update.

The HVP direction mixes a reduced direction v with a rigid motion of the kinematic
vertices, as the adjoint of a prescribed motion needs.
"""
import dataclasses
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


@functools.lru_cache(maxsize=None)
def _config1_second_iterate():
    sc = scenes.make_config(1)
    x0 = oracle.embed(sc, sc.iterate(0))
    a = oracle.accd(sc, x0, oracle.embed(sc, sc.dq(0), displacement=True))["alpha"]
    return scenes.with_second_iterate(sc, a)


def _gpu_state(sc, t, lag_t):
    from paper_2409_16385_gb300 import ContactScene
    cs = ContactScene(sc, pair_capacity=1 << 18, bsr_capacity=1 << 19, rec_capacity=1 << 22)
    q, qn = _t(sc.iterate(t)), _t(sc.iterate(lag_t))
    lag = cs.friction_lag(qn, cs.build_candidates(qn, out=cs.new_pairs())) if sc.params["mu"] > 0 else None
    pairs = cs.build_candidates(q)
    return cs, q, pairs, lag


def _oracle_state(sc, t, lag_t, pairs_gpu):
    x = oracle.embed(sc, sc.iterate(t))
    xn = oracle.embed(sc, sc.iterate(lag_t))
    lag = oracle.friction_lag(sc, xn, oracle.pairs(sc, xn)) if sc.params["mu"] > 0 else None
    h = pairs_gpu.host()
    prs = dict(type=h["type"], i=h["i"], j=h["j"])   # same list on both sides (set parity is tested elsewhere)
    return x, prs, lag


def _cases():
    return [("config1", _config1_second_iterate, 1, 0), ("bubble_small", lambda: scenes.make_config(2, small=True), 7, 6)]


@pytest.mark.parametrize("name,make,t,lag_t", _cases())
def test_hvp_matches_oracle(name, make, t, lag_t):
    sc = make()
    cs, q, pairs, lag = _gpu_state(sc, t, lag_t)
    x, prs, lago = _oracle_state(sc, t, lag_t, pairs)
    rng = np.random.default_rng(5)
    kin = sc.kinematic
    for kin_dir in (None, np.array([0.3, -0.2, 1.0])):
        v = rng.normal(size=(sc.Ns, 3))
        out, out_kin = cs.contact_hvp(q, pairs, _t(v), lag=lag, kin_dir=kin_dir)
        torch.cuda.synchronize()
        assert cs.status()["flags"] == 0
        u = oracle.embed(sc, v, displacement=True)
        if kin_dir is not None:
            u[kin] = kin_dir
        ro, rk = oracle.hvp(sc, x, prs, lago, u)
        g = out.cpu().numpy()
        scale = np.abs(ro).max()
        assert scale > 0
        assert np.abs(g - ro).max() <= TOL * scale, (name, np.abs(g - ro).max() / scale)
        gk = out_kin.cpu().numpy()
        if kin.any():
            assert np.abs(gk - rk).max() <= TOL * max(np.abs(rk).max(), 1e-300) + 1e-12 * scale


@pytest.mark.parametrize("name,make,t,lag_t", _cases())
def test_unprojected_hessian_matches_oracle(name, make, t, lag_t):
    sc = make()
    cs, q, pairs, lag = _gpu_state(sc, t, lag_t)
    x, prs, lago = _oracle_state(sc, t, lag_t, pairs)
    E, g, H = cs.eval_contact(q, pairs, lag, project=False)
    torch.cuda.synchronize()
    ro = oracle.eval_contact(sc, x, prs, lago, project=False)
    h = H.host()
    hg = {}
    for r in range(sc.Ns):
        for k in range(h["row_ptr"][r], h["row_ptr"][r + 1]):
            hg[(r, int(h["col"][k]))] = h["val"][k]
    ho = {(int(i), int(j)): vv for i, j, vv in zip(ro["I"], ro["J"], ro["V"])}
    assert set(hg) == set(ho)
    hs = max(np.abs(vv).max() for vv in ho.values())
    assert max(np.abs(hg[k] - ho[k]).max() for k in ho) <= TOL * hs
    # the HVP of the same state equals this matrix times v
    v = np.random.default_rng(9).normal(size=(sc.Ns, 3))
    out, _ = cs.contact_hvp(q, pairs, _t(v), lag=lag)
    ref = np.zeros_like(v)
    for (r, c), B in hg.items():
        ref[r] += B @ v[c]
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    # and the projected Hessian differs (some pair Hessians are indefinite)
    _, _, Hp = cs.eval_contact(q, pairs, lag)
    assert not np.array_equal(Hp.host()["val"], h["val"])


def test_hvp_is_bitwise_repeatable():
    sc = _config1_second_iterate()
    cs, q, pairs, lag = _gpu_state(sc, 1, 0)
    v = _t(np.random.default_rng(2).normal(size=(sc.Ns, 3)))
    outs = [cs.contact_hvp(q, pairs, v, lag=lag, kin_dir=(0.0, 0.0, 1.0)) for _ in range(3)]
    ref = (outs[0][0].cpu().numpy().tobytes(), outs[0][1].cpu().numpy().tobytes())
    for o in outs[1:]:
        assert (o[0].cpu().numpy().tobytes(), o[1].cpu().numpy().tobytes()) == ref


def test_set_kinematic_equals_a_scene_built_with_the_new_positions():
    from paper_2409_16385_gb300 import ContactScene
    sc = scenes.make_config(1)
    shift = np.array([0.0, 0.0, 1e-4])
    kin = sc.kinematic
    moved = dataclasses.replace(sc, x_kin=np.where(kin[:, None], sc.x_kin + shift, sc.x_kin))
    q = _t(sc.iterate(0))
    a = ContactScene(sc, pair_capacity=1 << 18, bsr_capacity=1 << 19, rec_capacity=1 << 22)
    b = ContactScene(moved, pair_capacity=1 << 18, bsr_capacity=1 << 19, rec_capacity=1 << 22)
    a.set_kinematic(_t(moved.x_kin))
    outs = []
    for cs in (a, b):
        pr = cs.build_candidates(q)
        E, g, H = cs.eval_contact(q, pr, None)
        ph = pr.host()
        outs.append((ph["i"].tobytes(), ph["j"].tobytes(), ph["d"].tobytes(), E.cpu().numpy().tobytes(),
                     g.cpu().numpy().tobytes(), H.host()["val"].tobytes()))
        assert cs.status()["flags"] == 0
    assert outs[0] == outs[1]
    assert len(a.build_candidates(q).host()["i"]) > 0
