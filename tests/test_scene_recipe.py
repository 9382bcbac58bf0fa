"""The seeded scene generators follow the stated workload recipes (CPU only).

Sizes, parameters and motions of the synthetic stand-ins for the paper's scenes:
- sphere on pad;
- bubble grasp (Sec. IV-A);
- plate in rack (Sec. IV-B);
- the batch of grasps;
- the pad-lift trajectory.
Where the paper prints a value (contact parameters and materials of Sec. IV-A), the
generator's value is checked against the fixture in tests/golden/.
"""
import functools
import json
import os

import numpy as np
import pytest

from paper_2409_16385_gb300 import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


@functools.lru_cache(maxsize=None)
def _cfg(k, small=False):
    return scenes.make_config(k, small=small)


def _paper():
    with open(GOLD) as f:
        return json.load(f)


def _embedding_is_barycentric(sc):
    emb = ~sc.kinematic
    w = sc.w[emb]
    assert np.all(w >= -1e-12) and np.allclose(w.sum(1), 1.0, atol=1e-13)
    # the rest cage reproduces the rest surface: each vertex inside its own tet
    tets = {tuple(t) for t in sc.cage_tets.tolist()}
    assert all(tuple(r) in tets for r in sc.cage_idx[emb].tolist())


def test_sphere_on_pad():
    sc = _cfg(1)
    assert (sc.Nv, sc.F, sc.E, sc.Ns, len(sc.cage_tets)) == (6787, 13312, 20096, 343, 1080)
    emb = ~sc.kinematic
    assert emb.sum() == 2562 and sc.kinematic.sum() == 4225
    assert (emb[sc.tris[:, 0]]).sum() == 5120
    _embedding_is_barycentric(sc)
    xr = scenes.embedded_positions(sc, sc.q_rest)
    r = np.linalg.norm(xr[emb] - xr[emb].mean(0), axis=1)
    assert np.allclose(r, 0.05, rtol=1e-12)
    assert np.all(sc.x_kin[sc.kinematic][:, 2] == 0.0)
    p = sc.params
    assert (p["dhat"], p["kappa"], p["mu"]) == (1e-3, 1e4, 0.5)
    q0 = sc.iterate(0)
    jitter = (q0 - sc.q_rest) - (q0 - sc.q_rest).mean(0)
    assert 0.9e-3 < jitter.std() < 1.1e-3                      # N(0, 1 mm) per node
    x0 = scenes.embedded_positions(sc, q0)
    assert abs(x0[emb][:, 2].min() - 0.3 * p["dhat"]) <= 1e-15  # 0.3 dhat above the pad
    dx = scenes.embedded_positions(sc, sc.dq(0))
    assert abs(np.linalg.norm(dx[emb], axis=1).max() - 5e-3) <= 1e-15


def test_bubble_grasp():
    sc = _cfg(2)
    sl = sc.node_slices
    assert sc.F == 100_820 + 2 * 40_500 and sc.Nv == 50_412 + 2 * 20_252
    nodes = {k: v.stop - v.start for k, v in sl.items()}
    assert 1400 <= nodes["body"] <= 1600 and 1900 <= nodes["top"] <= 2100 and 1900 <= nodes["bottom"] <= 2100
    assert sc.kinematic.sum() == 0
    _embedding_is_barycentric(sc)
    p = sc.params
    assert (p["dhat"], p["mu"]) == (5e-4, 0.8)
    assert sc.n_iterates == 60
    body = sc.body == 0
    top = sc.body == 1
    ymax = []
    for t in range(0, 60, 3):
        x = scenes.embedded_positions(sc, sc.iterate(t))
        ymax.append(x[body, 1].max())
        gap = x[top, 1].min() - ymax[-1]
        assert 0.2 * p["dhat"] - 1e-12 <= gap <= 0.8 * p["dhat"] + 1e-12
    # the top of the body moves in 1 mm per step (3 iterates), 2 cm over the 20 steps
    assert np.allclose(np.diff(ymax), -1e-3, atol=1e-12)


def test_plate_in_rack():
    sc = _cfg(3)
    tine = sc.kinematic[sc.tris[:, 0]]
    assert tine.sum() == 20 * 4000 and 55_000 <= (~tine).sum() <= 65_000
    assert sc.Ns == 800 and sc.n_iterates == 100
    assert sc.params["dhat"] == 2e-4
    _embedding_is_barycentric(sc)


def test_batched_grasps_sizes_and_cages():
    b = scenes.batched_grasp(n_scenes=32)
    tris = np.array([sc.F for sc, _ in b.parts])
    assert tris.min() >= 0.95 * 2000 and tris.max() <= 1.05 * 50_000
    # log-uniform sizes: the mean of log(size) near the middle of the log range
    assert abs(np.log(tris).mean() - 0.5 * (np.log(2000) + np.log(50_000))) < 0.5
    ratio = np.array([sc.Nv / sc.Ns for sc, _ in b.parts])
    assert 30 <= np.median(ratio) <= 50                        # about 1 node per 40 vertices
    for sc, _ in b.parts[:4]:
        _embedding_is_barycentric(sc)


def test_pad_lift_and_paper_materials():
    paper = _paper()
    sc = _cfg(5)
    assert sc.n_steps == 20 and sc.checkpoint_every == 5 and sc.theta == 1e-4
    assert sc.material == paper["materials"]["teddy"]
    phys = scenes.bubble_grasp_physical()
    assert phys.materials[0] == paper["materials"]["teddy"]
    assert phys.materials[1] == paper["materials"]["bubble"] == phys.materials[2]
    bg = paper["bubble_gripper"]
    assert (sc.params["kappa"], sc.params["eps_v"]) == (bg["kappa"], bg["eps_v"])
    assert sc.params["dhat"] == bg["dhat"]


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_generators_are_seeded(k):
    a = scenes.make_config(k, small=True)
    b = scenes.make_config(k, small=True)
    assert np.array_equal(a.iterate(0), b.iterate(0)) and np.array_equal(a.w, b.w)
    c = scenes.make_config(k, seed=1, small=True)
    assert not np.array_equal(a.iterate(0), c.iterate(0)) or k == 5
