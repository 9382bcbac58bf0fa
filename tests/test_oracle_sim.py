"""Pins of the oracle's reduced Newton driver and trajectory adjoint (CPU only).

Elasticity: the corotational energy against its defining properties (zero and stress
free at rest, rotation invariance, the small-strain limit of linear elasticity), the
first Piola-Kirchhoff stress against complex-step derivatives of the energy, the polar
rotation against numpy's SVD, the exact Hessian against central differences of the
stress.  Mass: total mass and weight against the enclosed volume.  Driver: the converged
step satisfies its optimality condition, lowers the incremental potential and leaves the
surfaces apart.  Adjoint: against central differences of the whole trajectory.
"""
import dataclasses
import functools

import numpy as np

import oracle
from oracle import sim
from paper_2409_16385_gb300 import scenes

MU, LAM = sim.lame(5e4, 0.45)


def _rot(rng):
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return Q * np.sign(np.linalg.det(Q))


def _F(rng, n=8, s=0.2):
    return np.stack([_rot(rng) @ (np.eye(3) + s * rng.normal(size=(3, 3))) for _ in range(n)])


def test_energy_is_zero_and_stress_free_at_rest_and_rotation_invariant():
    rng = np.random.default_rng(0)
    I = np.eye(3)[None]
    assert abs(sim.psi(I, MU, LAM)[0]) < 1e-20
    assert np.abs(sim.first_pk(I, MU, LAM)).max() < 1e-10
    F = _F(rng)
    Q = np.stack([_rot(rng) for _ in range(len(F))])
    assert np.allclose(sim.psi(Q @ F, MU, LAM), sim.psi(F, MU, LAM), rtol=1e-12, atol=0)
    assert np.allclose(sim.first_pk(Q @ F, MU, LAM), Q @ sim.first_pk(F, MU, LAM), rtol=1e-10, atol=1e-9)


def test_lame_parameters_give_back_youngs_modulus_and_poissons_ratio():
    """Uniaxial stretch by a small e with the lateral strain t free: the energy through the
    Lame parameters of (E, nu) is least at t = -nu e, and there it is E e^2 / 2 (the
    definitions of Poisson's ratio and Young's modulus), up to O(e) relative terms."""
    for E, nu in ((5e4, 0.45), (1e4, 0.3)):
        mu, lam = sim.lame(E, nu)
        e = 1e-5

        def energy(t):
            return sim.psi(np.diag([1.0 + e, 1.0 + t, 1.0 + t])[None], mu, lam)[0]

        ts = np.array([-e, 0.0, e])
        a, b, _ = np.polyfit(ts, [energy(t) for t in ts], 2)
        t_min = -b / (2.0 * a)
        assert np.isclose(-t_min / e, nu, rtol=1e-3), (E, nu, -t_min / e)
        assert np.isclose(2.0 * energy(t_min) / e ** 2, E, rtol=1e-3), (E, nu)


def test_polar_rotation_matches_the_svd():
    rng = np.random.default_rng(1)
    F = _F(rng, s=0.4)
    U, _, Vt = np.linalg.svd(F)
    R_svd = U @ Vt
    R = sim.polar_rotation(F)
    assert np.abs(R - R_svd).max() < 1e-13
    S = np.swapaxes(R, 1, 2) @ F
    assert np.abs(S - np.swapaxes(S, 1, 2)).max() < 1e-13
    assert np.all(np.linalg.eigvalsh(0.5 * (S + np.swapaxes(S, 1, 2))) > 0)


def test_small_strain_limit_is_linear_elasticity():
    rng = np.random.default_rng(2)
    G = rng.normal(size=(3, 3))
    for eps in (1e-3, 1e-4):
        F = np.eye(3) + eps * G
        e = 0.5 * (G + G.T) * eps
        lin = MU * np.sum(e * e) + 0.5 * LAM * np.trace(e) ** 2
        assert abs(sim.psi(F[None], MU, LAM)[0] - lin) <= 30 * eps * abs(lin)


def test_stress_is_the_complex_step_derivative_of_the_energy():
    rng = np.random.default_rng(3)
    F = _F(rng)
    P = sim.first_pk(F, MU, LAM)
    for _ in range(4):
        E = rng.normal(size=F.shape)
        d = sim.psi(F + 1e-30j * E, MU, LAM).imag / 1e-30
        assert np.allclose(d, np.einsum("tij,tij->t", P, E), rtol=1e-11, atol=1e-9)


def test_stress_differential_matches_central_differences():
    rng = np.random.default_rng(4)
    F = _F(rng)
    dF = rng.normal(size=F.shape)
    exact = sim.first_pk_differential(F, dF, MU, LAM)
    h = 1e-6
    fd = (sim.first_pk(F + h * dF, MU, LAM) - sim.first_pk(F - h * dF, MU, LAM)) / (2 * h)
    assert np.abs(exact - fd).max() <= 1e-6 * np.abs(exact).max()


@functools.lru_cache(maxsize=None)
def _model():
    sc = scenes.make_config(5, small=True)
    return sc, sim.build_model(sc)


def test_volumes_mass_and_weight():
    sc, m = _model()
    Vk = sim.vertex_volumes(sc)
    emb = ~sc.kinematic
    x = oracle.embed(sc, sc.q0)
    tri = sc.tris[emb[sc.tris[:, 0]]]
    # enclosed volume by the divergence theorem about the origin (a different split)
    vol = abs(np.einsum("ij,ij->i", x[tri[:, 0]], np.cross(x[tri[:, 1]], x[tri[:, 2]])).sum() / 6.0)
    assert abs(Vk.sum() - vol) <= 1e-12 * vol
    assert abs(vol - 4.0 / 3.0 * np.pi * 0.05 ** 3) < 0.1 * vol
    assert abs(m.V_T.sum() - vol) <= 1e-12 * vol
    rho = sc.material["rho"]
    assert abs(m.M.sum() - rho * vol) <= 1e-12 * rho * vol          # sum of weights is 1
    assert np.allclose(m.f_ext.sum(0), rho * vol * sc.gravity, rtol=1e-12)
    assert np.allclose(m.M, m.M.T) and np.linalg.eigvalsh(m.M).min() > -1e-15


def test_vertex_volumes_of_an_offset_octahedron():
    """The per-vertex split of the enclosed volume (one third of each incident triangle's
    cone to the body's centroid): a regular octahedron of radius r has eight congruent
    cones and four triangles at every vertex, so each of its six vertices takes
    (4/3) r^3 / 6, wherever the octahedron sits.  Each vertex is its own cage node here."""
    import types
    r, c = 0.3, np.array([3.0, -2.0, 5.0])
    X = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float) * r + c
    tris = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                     [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], np.int32)
    n = len(X)
    sc = types.SimpleNamespace(
        Nv=n, Ns=n, q0=X, x_kin=np.zeros((n, 3)), kinematic=np.zeros(n, bool), body=np.zeros(n, np.int64),
        tris=tris, cage_idx=np.repeat(np.arange(n, dtype=np.int32)[:, None], 4, axis=1),
        w=np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)))
    Vk = sim.vertex_volumes(sc)
    assert np.allclose(Vk, 4.0 / 3.0 * r ** 3 / 6.0, rtol=1e-12)


def test_reduced_mass_is_the_kinetic_energy_through_the_embedding():
    """M^q = J^T M J (Sec. III-D): for any reduced velocity v, v^T M^q v equals the lumped
    full-space kinetic form sum_k rho V_k |(J v)_k|^2, with J v taken by the embedding."""
    sc, m = _model()
    Vk = sim.vertex_volumes(sc)
    rho = sc.material["rho"]
    rng = np.random.default_rng(11)
    for _ in range(5):
        v = rng.normal(size=(sc.Ns, 3))
        xv = oracle.embed(sc, v, displacement=True)
        full = float(np.sum(rho * Vk[:, None] * xv * xv))
        assert abs(float(np.sum(v * (m.M @ v))) - full) <= 1e-12 * full


def test_free_flight_of_a_rigid_translation_is_exact():
    """Far from any contact and with every cage node free, a body translated rigidly and
    moving at constant velocity takes one backward-Euler step exactly
    (Sec. III-A): q^{n+1} = 2 q^n - q^{n-1} + h^2 g.  The elastic forces of a translation
    vanish, and J^T M J applied to a uniform field is J^T f_ext / g, since the weights sum
    to 1."""
    sc, m = _model()
    active = np.zeros(sc.Ns, bool)
    active[sc.cage_tets[m.V_T > 0].ravel()] = True
    m_free = dataclasses.replace(m, free=active)
    up = np.array([0.0, 0.0, 1.0])                   # a metre from the pad and its motion
    qp = sc.q0 + up
    vel = np.array([1e-3, -2e-3, 5e-4])
    q, it = sim.newton_step(m_free, qp, qp - vel, np.zeros(3), sc.params["kappa"], None)
    h = sc.params["h"]
    expect = qp + vel + h * h * sc.gravity
    assert it <= 3
    assert np.abs(q[active] - expect[active]).max() <= 1e-12


def test_elastic_gradient_and_hessian_match_central_differences():
    sc, m = _model()
    rng = np.random.default_rng(5)
    q = sc.q0 + 2e-3 * rng.normal(size=sc.q0.shape)
    v = rng.normal(size=q.shape)
    h = 1e-7
    g = sim.elastic_gradient(m, q)
    fd = (sim.elastic_energy(m, q + h * v) - sim.elastic_energy(m, q - h * v)) / (2 * h)
    assert abs(fd - np.sum(g * v)) <= 1e-6 * abs(np.sum(g * v))
    H = sim.elastic_hessian(m, q, project=False)
    fdg = (sim.elastic_gradient(m, q + h * v) - sim.elastic_gradient(m, q - h * v)) / (2 * h)
    assert np.abs(H @ v.ravel() - fdg.ravel()).max() <= 1e-6 * np.abs(fdg).max()
    assert np.allclose(H, H.T, rtol=0, atol=1e-9 * np.abs(H).max())
    Hp = sim.elastic_hessian(m, q, project=True)
    assert np.linalg.eigvalsh(Hp).min() > -1e-8 * np.abs(Hp).max()


def test_newton_step_converges_and_keeps_surfaces_apart():
    sc, m = _model()
    kappa = sc.params["kappa"]
    lag = sim.initial_lag(m, kappa)
    shift = sc.theta * sc.pad_dir
    q, it = sim.newton_step(m, sc.q0, sc.q0, shift, kappa, lag)
    assert it < 30
    sc1 = sim.shifted_scene(m, shift, kappa)
    phi, g, scale, x, _ = sim._evaluate(m, sc1, q, sc.q0, lag, False)
    assert np.abs(g[m.free]).max() <= 1e-12 * scale
    phi0, _, _, _, _ = sim._evaluate(m, sc1, sc.q0, sc.q0, lag, False)
    assert phi < phi0
    assert np.array_equal(q[~m.free], sc.q0[~m.free])
    assert oracle.intersection_free(sc1, x)
    assert len(oracle.pairs(sc1, x)["type"]) > 0


def test_adjoint_matches_central_differences_of_the_trajectory():
    sc, m = _model()
    kappa, theta, N = sc.params["kappa"], sc.theta, 3
    adj = sim.adjoint(m, theta, kappa, N)

    def L(th, k):
        qs, lag, _ = sim.trajectory(m, th, k, N)
        return sim.loss(m, qs[-1], th, k, lag, N)[0]

    h = 1e-7
    d_theta = (L(theta + h, kappa) - L(theta - h, kappa)) / (2 * h)
    d_kappa = (L(theta, kappa * (1 + 1e-3)) - L(theta, kappa * (1 - 1e-3))) / (2e-3 * kappa)
    assert adj["loss"] > 0
    assert abs(d_theta - adj["dtheta"]) <= 1e-6 * abs(adj["dtheta"])
    assert abs(d_kappa - adj["dkappa"]) <= 1e-6 * abs(adj["dkappa"])
