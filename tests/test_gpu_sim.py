"""GPU parity of the reduced Newton driver and of the trajectory adjoint.

The product driver (torch on the GPU + the CUDA contact stage) against the oracle driver
(numpy + the CPU contact oracle): cage elasticity, mass and weight, one time step, a short
trajectory; the autograd adjoint (HVP kernel + implicit steps + checkpointing) against
the oracle's adjoint and against central differences of the GPU trajectory.
"""
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
def _pair(small=True):
    from paper_2409_16385_gb300.sim import Simulator
    sc = scenes.make_config(5, small=small)
    return sc, Simulator(sc), osim.build_model(sc)


def test_model_matches_oracle():
    sc, s, m = _pair()
    assert np.allclose(s.elastic.V_T.cpu().numpy(), m.V_T, rtol=1e-12, atol=1e-18)
    assert np.allclose(s.M.cpu().numpy(), m.M, rtol=1e-12, atol=1e-16)
    assert np.allclose(s.f_ext.cpu().numpy(), m.f_ext, rtol=1e-12, atol=1e-15)
    assert np.array_equal(s.free.cpu().numpy(), m.free)


def test_elasticity_matches_oracle():
    sc, s, m = _pair()
    rng = np.random.default_rng(0)
    q = sc.q0 + 3e-3 * rng.normal(size=sc.q0.shape)
    v = rng.normal(size=q.shape)
    qd, vd = _t(q), _t(v)
    e_ref = osim.elastic_energy(m, q)
    assert abs(float(s.elastic.energy(qd)) - e_ref) <= 1e-11 * abs(e_ref)
    g_ref = osim.elastic_gradient(m, q)
    assert np.abs(s.elastic.gradient(qd).cpu().numpy() - g_ref).max() <= 1e-10 * np.abs(g_ref).max()
    H = osim.elastic_hessian(m, q, project=False)
    hv_ref = (H @ v.ravel()).reshape(-1, 3)
    hv = s.elastic.hvp(qd, vd).cpu().numpy()
    assert np.abs(hv - hv_ref).max() <= 1e-9 * np.abs(hv_ref).max()
    Hd = s.elastic.assemble_dense(s.elastic.tet_hessians(qd, False)).cpu().numpy()
    assert np.abs(Hd - H).max() <= 1e-9 * np.abs(H).max()
    Hp = s.elastic.assemble_dense(s.elastic.tet_hessians(qd, True)).cpu().numpy()
    assert np.linalg.eigvalsh(Hp).min() > -1e-8 * np.abs(Hp).max()


def test_one_step_matches_oracle():
    sc, s, m = _pair()
    kappa = sc.params["kappa"]
    shift = sc.theta * sc.pad_dir
    lag_o = osim.initial_lag(m, kappa)
    q_o, _ = osim.newton_step(m, sc.q0, sc.q0, shift, kappa, lag_o)
    lag_g = s.initial_lag(kappa)
    q_g, info = s.step(s.q0, s.q0, _t(shift), kappa, lag_g)
    # converged: either below rtol = 1e-12, or stopped by a step below four ulps, which
    # leaves the residual at its rounding floor (a few 1e-13 to about 1e-12 of the largest
    # force term); the state itself is held to the 1e-9 parity bar below
    assert info.reason in ("residual", "step") and info.iterations < 40, info
    assert info.residual <= (1e-12 if info.reason == "residual" else 1e-10), info
    d = np.abs(q_g.cpu().numpy() - q_o).max()
    assert d <= 1e-9 * np.abs(q_o - sc.q0).max(), d


def test_trajectory_matches_oracle():
    sc, s, m = _pair()
    kappa, theta, N = sc.params["kappa"], sc.theta, 5
    qs_o, lag_o, _ = osim.trajectory(m, theta, kappa, N)
    qs_g, lag_g, infos = s.trajectory(theta, kappa, N)
    assert all(i.converged for i in infos), infos
    for n in range(1, N + 1):
        ref = qs_o[n]
        assert np.abs(qs_g[n].cpu().numpy() - ref).max() <= 1e-8 * np.abs(ref - sc.q0).max(), n
    L_o, g_o = osim.loss(m, qs_o[N], theta, kappa, lag_o, N)
    g_g = s.contact_force(qs_g[N], _t(N * theta * sc.pad_dir), kappa, lag_g).cpu().numpy()
    assert np.abs(g_g - g_o).max() <= 1e-7 * np.abs(g_o).max()


def _grads(s, theta, kappa, N, k, solver="dense"):
    from paper_2409_16385_gb300.adjoint import trajectory_loss
    th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    ka = torch.tensor(kappa, dtype=torch.float64, device="cuda", requires_grad=True)
    L = trajectory_loss(s, th, ka, N, k, solver=solver)
    L.backward()
    return float(L), float(th.grad), float(ka.grad)


def _loss(s, theta, kappa, N):
    from paper_2409_16385_gb300.adjoint import trajectory_loss
    with torch.no_grad():
        return float(trajectory_loss(s, torch.tensor(theta, dtype=torch.float64, device="cuda"),
                                     torch.tensor(kappa, dtype=torch.float64, device="cuda"), N, 0))


def test_adjoint_matches_oracle_and_central_differences_small():
    sc, s, m = _pair()
    kappa, theta, N = sc.params["kappa"], sc.theta, 6
    L, d_theta, d_kappa = _grads(s, theta, kappa, N, k=2)
    ref = osim.adjoint(m, theta, kappa, N)
    assert abs(L - ref["loss"]) <= 1e-8 * ref["loss"]
    assert abs(d_theta - ref["dtheta"]) <= 1e-6 * abs(ref["dtheta"])
    assert abs(d_kappa - ref["dkappa"]) <= 1e-6 * abs(ref["dkappa"])
    h = 1e-7
    fd_theta = (_loss(s, theta + h, kappa, N) - _loss(s, theta - h, kappa, N)) / (2 * h)
    fd_kappa = (_loss(s, theta, kappa * (1 + 1e-3), N) - _loss(s, theta, kappa * (1 - 1e-3), N)) / (2e-3 * kappa)
    assert abs(fd_theta - d_theta) <= 1e-6 * abs(d_theta)
    assert abs(fd_kappa - d_kappa) <= 1e-6 * abs(d_kappa)


def test_matrix_free_adjoint_equals_dense():
    sc, s, m = _pair()
    kappa, theta, N = sc.params["kappa"], sc.theta, 4
    a = _grads(s, theta, kappa, N, k=2, solver="dense")
    b = _grads(s, theta, kappa, N, k=2, solver="minres")
    assert abs(a[1] - b[1]) <= 1e-8 * abs(a[1])
    assert abs(a[2] - b[2]) <= 1e-8 * abs(a[2])


def test_checkpointing_does_not_change_the_gradient():
    sc, s, m = _pair()
    kappa, theta, N = sc.params["kappa"], sc.theta, 4
    a = _grads(s, theta, kappa, N, k=0)
    b = _grads(s, theta, kappa, N, k=1)
    assert abs(a[1] - b[1]) <= 1e-10 * abs(a[1]) and abs(a[2] - b[2]) <= 1e-10 * abs(a[2])


@pytest.mark.slow
def test_adjoint_full_config5_matches_central_differences():
    """The full config-5 scene: 20 steps, checkpoints every 5."""
    sc, s, m = _pair(small=False)
    kappa, theta, N = sc.params["kappa"], sc.theta, sc.n_steps
    L, d_theta, d_kappa = _grads(s, theta, kappa, N, k=sc.checkpoint_every)
    h = 1e-7
    fd_theta = (_loss(s, theta + h, kappa, N) - _loss(s, theta - h, kappa, N)) / (2 * h)
    fd_kappa = (_loss(s, theta, kappa * (1 + 1e-3), N) - _loss(s, theta, kappa * (1 - 1e-3), N)) / (2e-3 * kappa)
    assert L > 0
    assert abs(fd_theta - d_theta) <= 1e-6 * abs(d_theta), (fd_theta, d_theta)
    assert abs(fd_kappa - d_kappa) <= 1e-6 * abs(d_kappa), (fd_kappa, d_kappa)
