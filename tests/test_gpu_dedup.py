"""GPU parity of the deduplicated contact set (EIPC_PARAM_DEDUP) and of the contact stage
evaluated on it: identical (type, i, j) lists against oracle.dedup (outside the dhat band),
E, g_r and H_r within 1e-9 (the same bars as the literal set)."""
import functools

import numpy as np
import pytest

import oracle
from paper_2409_16385_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@functools.lru_cache(maxsize=None)
def _scene(k, small):
    return scenes.make_config(k, small=small)


@pytest.mark.parametrize("k,small,t", [(1, False, 0), (2, True, 7), (3, True, 11)])
def test_dedup_pairs_and_evaluation_match_oracle(k, small, t):
    from paper_2409_16385_gb300 import ContactScene
    sc = _scene(k, small)
    t = min(t, sc.n_iterates - 1)
    lag_t = sc.lag_of(t)
    cs = ContactScene(sc, pair_capacity=1 << 20, bsr_capacity=1 << 21, rec_capacity=1 << 23)
    cs.set_dedup(True)
    q, qn = _t(sc.iterate(t)), _t(sc.iterate(lag_t))
    pn = cs.build_candidates(qn, out=cs.new_pairs())
    lag = cs.friction_lag(qn, pn) if sc.params["mu"] > 0 else None
    pairs = cs.build_candidates(q)
    E, g, H = cs.eval_contact(q, pairs, lag)
    torch.cuda.synchronize()
    assert cs.status()["flags"] == 0
    x, xn = oracle.embed(sc, sc.iterate(t)), oracle.embed(sc, sc.iterate(lag_t))
    po = oracle.dedup(sc, x, oracle.pairs(sc, x))
    pon = oracle.dedup(sc, xn, oracle.pairs(sc, xn))
    hg = pairs.host()
    kg = list(zip(hg["type"].tolist(), hg["i"].tolist(), hg["j"].tolist()))
    ko = list(zip(po["type"].tolist(), po["i"].tolist(), po["j"].tolist()))
    assert kg == sorted(kg)
    dh = sc.params["dhat"]
    dg = dict(zip(kg, hg["d"].tolist())); do = dict(zip(ko, po["d"].tolist()))
    for key in set(kg) ^ set(ko):
        dk = dg.get(key, do.get(key))
        assert abs(dk - dh) <= 1e-12 * dh, (key, dk)
    cs.set_dedup(False)
    n_lit = int(cs.build_candidates(q).count.item())
    cs.set_dedup(True)
    assert len(kg) < n_lit
    lo = oracle.friction_lag(sc, xn, pon) if sc.params["mu"] > 0 else None
    ro = oracle.eval_contact(sc, x, po, lo)
    assert abs(float(E.item()) - ro["E"]) <= 1e-9 * abs(ro["E"])
    gg = g.cpu().numpy()
    assert np.abs(gg - ro["g"]).max() <= 1e-9 * np.abs(ro["g"]).max()
    h = H.host()
    hd = {}
    for r in range(sc.Ns):
        for kk in range(h["row_ptr"][r], h["row_ptr"][r + 1]):
            hd[(r, int(h["col"][kk]))] = h["val"][kk]
    ho = {(int(a), int(b)): v for a, b, v in zip(ro["I"], ro["J"], ro["V"])}
    assert set(hd) == set(ho)
    hs = max(np.abs(v).max() for v in ho.values())
    assert max(np.abs(hd[key] - ho[key]).max() for key in ho) <= 1e-9 * hs
