"""The reduced Newton driver with the sparse solve: the library's BSR SpMV against a dense
product, the block-Jacobi PCG Newton step against the dense one, and the physically
simulated bubble grasp (membranes' outer cage layers position-controlled, body and
membranes elastic under gravity, friction lagged every step) against the oracle driver."""
import functools

import numpy as np
import pytest

import oracle
from oracle import sim as osim
from paper_2409_16385_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@functools.lru_cache(maxsize=None)
def _physical_small():
    return scenes.bubble_grasp_physical(small=True)


def test_bsr_spmv_matches_dense():
    from paper_2409_16385_gb300 import ContactScene, bsr_spmv
    sc = scenes.make_config(2, small=True)
    cs = ContactScene(sc, pair_capacity=1 << 18, bsr_capacity=1 << 20, rec_capacity=1 << 22)
    q = _t(sc.iterate(5))
    _, _, H = cs.eval_contact(q, cs.build_candidates(q), None)
    nnzb = int(H.nnzb.item())
    x = _t(np.random.default_rng(0).normal(size=(sc.Ns, 3)))
    y0 = _t(np.random.default_rng(1).normal(size=(sc.Ns, 3)))
    y = bsr_spmv(H.row_ptr, H.col, H.val[:nnzb], x, out=y0.clone(), alpha=0.7, beta=-1.5)
    h = H.host()
    D = np.zeros((3 * sc.Ns, 3 * sc.Ns))
    for r in range(sc.Ns):
        for k in range(h["row_ptr"][r], h["row_ptr"][r + 1]):
            c = int(h["col"][k])
            D[3 * r:3 * r + 3, 3 * c:3 * c + 3] = h["val"][k]
    ref = 0.7 * (D @ x.cpu().numpy().ravel()) - 1.5 * y0.cpu().numpy().ravel()
    assert np.abs(y.cpu().numpy().ravel() - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("which", ["pad_lift", "grasp"])
def test_pcg_step_matches_dense_step(which):
    from paper_2409_16385_gb300.sim import Simulator
    sc = scenes.make_config(5, small=True) if which == "pad_lift" else _physical_small()
    a = Simulator(sc, solver="dense")
    b = Simulator(sc, solver="pcg")
    kappa = sc.params["kappa"]
    shift = torch.zeros(3, dtype=torch.float64, device="cuda")
    if which == "pad_lift":
        shift = sc.theta * a.pad_dir
    qa, ia = a.step(a.q0, a.q0, shift, kappa, a.initial_lag(kappa), q_fixed=a.prescribed(1))
    qb, ib = b.step(b.q0, b.q0, shift, kappa, b.initial_lag(kappa), q_fixed=b.prescribed(1))
    # both stop at this scene's rounding floor (a few 1e-11 of the largest force term)
    assert ia.converged and ib.converged, (ia, ib)
    assert ia.residual <= 1e-10 and ib.residual <= 1e-10, (ia, ib)
    assert ib.krylov_iterations > 0
    d = (qa - a.q0).abs().max()
    assert float((qa - qb).abs().max()) <= 1e-8 * float(d)


def test_physical_grasp_matches_oracle():
    from paper_2409_16385_gb300.sim import Simulator
    sc = _physical_small()
    s = Simulator(sc, solver="pcg")
    qs, _, infos = s.trajectory(0.0, sc.params["kappa"], 2)
    m = osim.build_model(sc)
    qo, _, _ = osim.trajectory(m, 0.0, sc.params["kappa"], 2)
    for n in (1, 2):
        ref = qo[n]
        assert np.abs(qs[n].cpu().numpy() - ref).max() <= 1e-8 * np.abs(ref - sc.q0).max(), n
    x = oracle.embed(sc, qs[2].cpu().numpy())
    assert oracle.intersection_free(sc, x)
    assert all(i.converged and i.residual <= 1e-10 for i in infos), infos
