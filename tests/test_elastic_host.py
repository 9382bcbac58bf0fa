"""The driver's cage elasticity (torch) against the oracle's, on CPU tensors (CPU only).

The torch module is device-agnostic: the same closed-form polar decomposition, stress,
exact stress differential and per-tet Hessians run here on CPU tensors. It is checked
against the oracle's numpy restatement, which computes the polar rotation by the rational
iteration and the Hessian by complex-step differentiation. This check has no GPU or CUDA
contact stage in the loop; the GPU run of the same comparison is in test_gpu_sim.py.
"""
import functools

import numpy as np
import pytest

from oracle import sim as osim
from paper_2409_16385_gb300 import scenes

torch = pytest.importorskip("torch")


@functools.lru_cache(maxsize=None)
def _setup():
    from paper_2409_16385_gb300.elastic import CorotationalCage
    sc = scenes.make_config(5, small=True)
    m = osim.build_model(sc)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64)
    cage = CorotationalCage(torch.tensor(sc.cage_tets), t(sc.q0), t(m.V_T), t(m.mu), t(m.lam))
    return sc, m, cage, t


def test_energy_gradient_and_hessians_match_the_oracle():
    sc, m, cage, t = _setup()
    rng = np.random.default_rng(2)
    q = sc.q0 + 3e-3 * rng.normal(size=sc.q0.shape)
    v = rng.normal(size=q.shape)
    e_ref = osim.elastic_energy(m, q)
    assert abs(float(cage.energy(t(q))) - e_ref) <= 1e-11 * abs(e_ref)
    g_ref = osim.elastic_gradient(m, q)
    assert np.abs(cage.gradient(t(q)).numpy() - g_ref).max() <= 1e-10 * np.abs(g_ref).max()
    H = osim.elastic_hessian(m, q, project=False)
    hv = cage.hvp(t(q), t(v)).numpy().ravel()
    assert np.abs(hv - H @ v.ravel()).max() <= 1e-9 * np.abs(H @ v.ravel()).max()
    Hd = cage.assemble_dense(cage.tet_hessians(t(q), False)).numpy()
    assert np.abs(Hd - H).max() <= 1e-9 * np.abs(H).max()
    # the driver clamps each tet's 9 x 9 Hessian in F, the oracle its 12 x 12 one in the
    # node positions: both PSD, equal where nothing is clamped (at rest below)
    Hp = cage.assemble_dense(cage.tet_hessians(t(q), True)).numpy()
    assert np.linalg.eigvalsh(Hp).min() > -1e-8 * np.abs(Hp).max()
    H0 = osim.elastic_hessian(m, sc.q0, project=False)
    Hp0 = cage.assemble_dense(cage.tet_hessians(t(sc.q0), True)).numpy()
    assert np.abs(Hp0 - H0).max() <= 1e-9 * np.abs(H0).max()


def test_block_assembly_equals_the_dense_one():
    sc, m, cage, t = _setup()
    q = t(sc.q0 + 1e-3 * np.random.default_rng(4).normal(size=sc.q0.shape))
    Ht = cage.tet_hessians(q, True)
    row_ptr, col, slot = cage.block_pattern()
    vals = cage.assemble_blocks(Ht, slot, len(col)).numpy()
    dense = np.zeros((3 * cage.ns, 3 * cage.ns))
    rp, cl = row_ptr.numpy(), col.numpy()
    for I in range(cage.ns):
        for k in range(rp[I], rp[I + 1]):
            J = cl[k]
            dense[3 * I:3 * I + 3, 3 * J:3 * J + 3] = vals[k]
    assert np.array_equal(dense != 0, cage.assemble_dense(Ht).numpy() != 0)
    assert np.abs(dense - cage.assemble_dense(Ht).numpy()).max() <= 1e-12 * np.abs(dense).max()
    assert np.all(np.diff(rp) > 0) and all(np.all(np.diff(cl[rp[I]:rp[I + 1]]) > 0) for I in range(cage.ns))


@pytest.mark.parametrize("phys", [False, True])
def test_vertex_volumes_match_the_oracle(phys):
    """Per-vertex volumes (cones of each vertex's triangles to its body's centroid) of the
    driver against the oracle's, on the pad-lift scene and on the three-body grasp."""
    from paper_2409_16385_gb300.sim import _vertex_volumes
    import oracle
    sc = scenes.bubble_grasp_physical(small=True) if phys else scenes.make_config(5, small=True)
    x = oracle.embed(sc, sc.q0)
    V = _vertex_volumes(sc, torch.tensor(x)).numpy()
    Vo = osim.vertex_volumes(sc)
    assert np.abs(V - Vo).max() <= 1e-12 * np.abs(Vo).max()
    assert np.all(V[sc.kinematic] == 0.0)


def test_lame_parameters_match_the_oracle():
    """The driver's (E, nu) -> (mu, lambda) conversion against the oracle's, which is pinned
    on Young's modulus and Poisson's ratio of a uniaxial stretch."""
    from paper_2409_16385_gb300.elastic import lame
    for E, nu in ((5e4, 0.45), (1e4, 0.3), (2e6, 0.0)):
        assert np.allclose(lame(E, nu), osim.lame(E, nu), rtol=1e-15, atol=0)
