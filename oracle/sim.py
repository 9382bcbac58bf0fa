"""Test infrastructure: CPU oracle of the reduced Newton driver and of the trajectory
adjoint built on the contact stage.

Written from the paper (arxiv 2409.16385) in plain numpy with dense matrices:
  * cage elasticity Phi(q) = sum_T V_T Psi(F_T), F_T = D_T (D_T^0)^{-1}, with V_T the sum of
    the per-vertex volumes V_k of the embedded vertices in T (Sec. III-D);
    Psi = linear corotational, mu ||F - R||^2 + lambda/2 (tr(R^T F) - 3)^2 (the model of
    Sec. IV-A), R the rotation of the polar decomposition F = R S;
  * reduced mass M^q = J^T M J with the lumped full-space mass rho V_k per vertex, and the
    generalised external force J^T f_ext (Sec. III-A, III-D);
  * the incremental potential E_IP(q) = 1/2 (q - q^n - h qdot^n)^T M^q (q - ...) +
    h^2 (Phi(q) + E_ext(q) + B(Jq) + D(Jq))  (Sec. III-A, III-B), minimised by projected
    Newton with the CCD step bound and backtracking (Sec. III-C);
  * the adjoint of a trajectory of such steps by implicit differentiation of each step's
    optimality condition, with the exact (unprojected) Hessians.
Readings where the paper is silent (per-vertex volume of a surface-only mesh, the sign of
E_ext, the lag state of a differentiated trajectory) follow the project's design notes.
The exact elastic Hessian is taken by complex-step differentiation of the first
Piola-Kirchhoff stress, with the polar rotation computed by the rational iteration
R <- (R + R^{-T}) / 2, which is analytic in F.  Only tests may import this module; it
shares nothing with the CUDA library or the product driver.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, Optional

import numpy as np

from . import accd, embed, eval_contact, friction_lag, hvp, pairs


def lame(E: float, nu: float):
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def _inv_transpose(A: np.ndarray) -> np.ndarray:
    """A^{-T} of a batch of 3 x 3 matrices: cofactor matrix / determinant."""
    c = np.empty_like(A)
    c[..., 0, 0] = A[..., 1, 1] * A[..., 2, 2] - A[..., 1, 2] * A[..., 2, 1]
    c[..., 0, 1] = A[..., 1, 2] * A[..., 2, 0] - A[..., 1, 0] * A[..., 2, 2]
    c[..., 0, 2] = A[..., 1, 0] * A[..., 2, 1] - A[..., 1, 1] * A[..., 2, 0]
    c[..., 1, 0] = A[..., 0, 2] * A[..., 2, 1] - A[..., 0, 1] * A[..., 2, 2]
    c[..., 1, 1] = A[..., 0, 0] * A[..., 2, 2] - A[..., 0, 2] * A[..., 2, 0]
    c[..., 1, 2] = A[..., 0, 1] * A[..., 2, 0] - A[..., 0, 0] * A[..., 2, 1]
    c[..., 2, 0] = A[..., 0, 1] * A[..., 1, 2] - A[..., 0, 2] * A[..., 1, 1]
    c[..., 2, 1] = A[..., 0, 2] * A[..., 1, 0] - A[..., 0, 0] * A[..., 1, 2]
    c[..., 2, 2] = A[..., 0, 0] * A[..., 1, 1] - A[..., 0, 1] * A[..., 1, 0]
    det = np.einsum("...j,...j->...", A[..., 0, :], c[..., 0, :])
    return c / det[..., None, None]


def polar_rotation(F: np.ndarray, max_iters: int = 80) -> np.ndarray:
    """R of F = R S for a batch [..., 3, 3] (real or complex): iterate until the real part
    stops changing, then three more rounds so a complex-step part has converged too."""
    R = np.array(F, copy=True)
    extra = 3
    for _ in range(max_iters):
        Rn = 0.5 * (R + _inv_transpose(R))
        done = np.abs((Rn - R).real).max() <= 1e-15 * max(1.0, np.abs(Rn.real).max())
        R = Rn
        if done:
            extra -= 1
            if extra < 0:
                break
    return R


def psi(F: np.ndarray, mu, lam) -> np.ndarray:
    """mu, lam: numbers or one value per matrix of the batch."""
    R = polar_rotation(F)
    D = F - R
    tr = np.einsum("...ij,...ij->...", R, F)        # tr(R^T F)
    return mu * np.einsum("...ij,...ij->...", D, D) + 0.5 * lam * (tr - 3.0) ** 2


def first_pk(F: np.ndarray, mu, lam) -> np.ndarray:
    R = polar_rotation(F)
    tr = np.einsum("...ij,...ij->...", R, F)
    mu3 = np.asarray(mu)[..., None, None]
    return 2.0 * mu3 * (F - R) + (np.asarray(lam) * (tr - 3.0))[..., None, None] * R


def first_pk_differential(F: np.ndarray, dF: np.ndarray, mu: float, lam: float, step: float = 1e-30) -> np.ndarray:
    """dP[dF] by complex step: Im P(F + i step dF) / step (exact to rounding)."""
    return first_pk(F + 1j * step * dF, mu, lam).imag / step


def vertex_volumes(sc) -> np.ndarray:
    """Per-vertex volume of each embedded closed surface: the cone of every triangle to
    its body's centroid, split equally among its three vertices (sums to the enclosed
    volume); zero on kinematic vertices."""
    x = embed(sc, sc.q0)
    V = np.zeros(sc.Nv)
    kin = sc.kinematic
    for b in np.unique(sc.body):
        members = sc.body == b
        if kin[members].all():
            continue
        tri = sc.tris[members[sc.tris[:, 0]]]
        c = x[members].mean(0)
        a, bb, cc = x[tri[:, 0]] - c, x[tri[:, 1]] - c, x[tri[:, 2]] - c
        vol = np.einsum("ij,ij->i", a, np.cross(bb, cc)) / 6.0
        if vol.sum() < 0:
            vol = -vol
        for k in range(3):
            np.add.at(V, tri[:, k], vol / 3.0)
    return V


@dataclasses.dataclass
class Model:
    """Everything the driver needs that does not change along a trajectory."""
    sc: object
    mu: np.ndarray           # [T] Lame parameters per tet
    lam: np.ndarray
    h: float
    Dm_inv: np.ndarray       # [T,3,3]
    V_T: np.ndarray          # [T]
    M: np.ndarray            # [Ns,Ns] scalar reduced mass (times I3 per component)
    f_ext: np.ndarray        # [Ns,3] generalised external force
    free: np.ndarray         # bool [Ns]


def build_model(sc) -> Model:
    """Materials: sc.materials (body id -> E, nu, rho; a tet takes the body of the vertices
    inside it) or one sc.material.  Dirichlet nodes: sc.prescribed_nodes or sc.fixed_nodes."""
    tets = sc.cage_tets
    q0 = sc.q0
    Dm = np.stack([q0[tets[:, 1]] - q0[tets[:, 0]], q0[tets[:, 2]] - q0[tets[:, 0]],
                   q0[tets[:, 3]] - q0[tets[:, 0]]], axis=2)
    Dm_inv = np.linalg.inv(Dm)
    Vk = vertex_volumes(sc)
    # tet of each embedded vertex: its cage_idx row is that tet's node list
    where = {tuple(t): i for i, t in enumerate(tets.tolist())}
    V_T = np.zeros(len(tets))
    emb = ~sc.kinematic
    mats = getattr(sc, "materials", None)
    tet_body = np.zeros(len(tets), np.int64)
    for k in np.nonzero(emb)[0]:
        t = where[tuple(sc.cage_idx[k].tolist())]
        V_T[t] += Vk[k]
        tet_body[t] = sc.body[k]

    def mat(b):
        return mats[int(b)] if mats else sc.material

    E = np.array([mat(b)["E"] for b in tet_body])
    nu = np.array([mat(b)["nu"] for b in tet_body])
    mu, lam = lame(E, nu)
    M = np.zeros((sc.Ns, sc.Ns))
    f = np.zeros((sc.Ns, 3))
    for k in np.nonzero(emb)[0]:
        idx, w = sc.cage_idx[k], sc.w[k]
        m = mat(sc.body[k])["rho"] * Vk[k]
        M[np.ix_(idx, idx)] += m * np.outer(w, w)
        f[idx] += m * w[:, None] * sc.gravity[None, :]
    active = np.zeros(sc.Ns, bool)
    active[tets[V_T > 0].ravel()] = True
    fixed = getattr(sc, "prescribed_nodes", None)
    if fixed is None:
        fixed = sc.fixed_nodes
    return Model(sc=sc, mu=mu, lam=lam, h=sc.params["h"], Dm_inv=Dm_inv, V_T=V_T, M=M, f_ext=f,
                 free=active & ~fixed)


def _deformation(m: Model, q: np.ndarray) -> np.ndarray:
    t = m.sc.cage_tets
    Ds = np.stack([q[t[:, 1]] - q[t[:, 0]], q[t[:, 2]] - q[t[:, 0]], q[t[:, 3]] - q[t[:, 0]]], axis=2)
    return Ds @ m.Dm_inv


def _scatter_tet_forces(m: Model, G: np.ndarray) -> np.ndarray:
    """Per-tet dE/dDs [T,3,3] (columns = nodes 1..3) -> nodal forces [Ns,3]."""
    t = m.sc.cage_tets
    out = np.zeros((m.sc.Ns, 3), dtype=G.dtype)
    for a in range(3):
        np.add.at(out, t[:, a + 1], G[:, :, a])
    np.add.at(out, t[:, 0], -G.sum(axis=2))
    return out


def elastic_energy(m: Model, q: np.ndarray) -> float:
    return float(np.sum(m.V_T * psi(_deformation(m, q), m.mu, m.lam)))


def elastic_gradient(m: Model, q: np.ndarray) -> np.ndarray:
    P = first_pk(_deformation(m, q), m.mu, m.lam)
    G = m.V_T[:, None, None] * (P @ np.swapaxes(m.Dm_inv, 1, 2))
    return _scatter_tet_forces(m, G)


def elastic_tet_hessians(m: Model, q: np.ndarray) -> np.ndarray:
    """Exact 12 x 12 Hessian of V_T Psi(F_T) per tet, node-major (3 a + c)."""
    F = _deformation(m, q)
    T = len(F)
    H = np.zeros((T, 12, 12))
    DmT = np.swapaxes(m.Dm_inv, 1, 2)
    for a in range(4):
        for c in range(3):
            dDs = np.zeros((T, 3, 3))
            if a == 0:
                dDs[:, c, :] = -1.0
            else:
                dDs[:, c, a - 1] = 1.0
            dP = first_pk_differential(F, dDs @ m.Dm_inv, m.mu, m.lam)
            G = m.V_T[:, None, None] * (dP @ DmT)            # d(dE/dDs)
            col = 3 * a + c
            for b in range(3):
                H[:, 3 * (b + 1):3 * (b + 1) + 3, col] = G[:, :, b]
            H[:, 0:3, col] = -G.sum(axis=2)
    return 0.5 * (H + np.swapaxes(H, 1, 2))


def _assemble_tets(m: Model, Ht: np.ndarray) -> np.ndarray:
    n = 3 * m.sc.Ns
    H = np.zeros((n, n))
    t = m.sc.cage_tets
    dofs = (3 * t[:, :, None] + np.arange(3)[None, None, :]).reshape(len(t), 12)
    for e in range(len(t)):
        H[np.ix_(dofs[e], dofs[e])] += Ht[e]
    return H


def elastic_hessian(m: Model, q: np.ndarray, project: bool) -> np.ndarray:
    Ht = elastic_tet_hessians(m, q)
    if project:
        lam_, V = np.linalg.eigh(Ht)
        Ht = np.einsum("tij,tj,tkj->tik", V, np.maximum(lam_, 0.0), V)
    return _assemble_tets(m, Ht)


def _blocks_to_dense(ns: int, r: dict) -> np.ndarray:
    H = np.zeros((3 * ns, 3 * ns))
    for I, J, B in zip(r["I"], r["J"], r["V"]):
        H[3 * I:3 * I + 3, 3 * J:3 * J + 3] += B
    return H


# ------------------------------------------------------------------ one time step
def shifted_scene(m: Model, shift: np.ndarray, kappa: float):
    sc = m.sc
    kin = sc.kinematic
    params = dict(sc.params, kappa=float(kappa))
    return dataclasses.replace(sc, x_kin=np.where(kin[:, None], sc.x_kin + shift, sc.x_kin), params=params)


def contact(sc_n, q: np.ndarray, lag, project: bool = True):
    x = embed(sc_n, q)
    prs = pairs(sc_n, x)
    r = eval_contact(sc_n, x, prs, lag, project=project)
    return x, prs, r


def _evaluate(m: Model, sc_n, q, q_tilde, lag, hessian: bool):
    """E_IPC, its gradient, a force scale for the stopping test, and optionally the
    projected-Newton Hessian."""
    x, prs, r = contact(sc_n, q, lag, project=True)
    h2 = m.h ** 2
    d = q - q_tilde
    Md = m.M @ d
    ge = elastic_gradient(m, q)
    phi = 0.5 * float(np.sum(d * Md)) + h2 * (elastic_energy(m, q) - float(np.sum(m.f_ext * q)) + r["E"])
    g = Md + h2 * (ge - m.f_ext + r["g"])
    scale = float((np.abs(Md) + h2 * (np.abs(ge) + np.abs(m.f_ext) + np.abs(r["g"])))[m.free].max())
    H = None
    if hessian:
        # the exact Hessian where it is positive definite on the free DoFs (quadratic
        # convergence), the projected-Newton one otherwise
        free3 = np.repeat(m.free, 3)
        _, _, r_exact = contact(sc_n, q, lag, project=False)
        H = np.kron(m.M, np.eye(3)) + h2 * (elastic_hessian(m, q, False) + _blocks_to_dense(sc_n.Ns, r_exact))
        try:
            np.linalg.cholesky(H[np.ix_(free3, free3)])
        except np.linalg.LinAlgError:
            H = np.kron(m.M, np.eye(3)) + h2 * (elastic_hessian(m, q, True) + _blocks_to_dense(sc_n.Ns, r))
    return phi, g, scale, x, H


def newton_step(m: Model, q_prev, q_prev2, shift, kappa, lag, rtol: float = 1e-12, max_iter: int = 100,
                q_fixed=None):
    """q^{n+1} = argmin E_IPC by projected Newton with the CCD step bound and backtracking,
    until the free residual is below rtol times the largest force term (its rounding floor
    is a few 1e-13) or the step is below four ulps of the positions.  Returns
    (q, iterations)."""
    sc_n = shifted_scene(m, shift, kappa)
    q_tilde = 2.0 * q_prev - q_prev2
    q = q_prev.copy()
    if q_fixed is not None:
        q[~m.free] = q_fixed[~m.free]
    free3 = np.repeat(m.free, 3)
    for it in range(max_iter):
        phi, g, scale, x, H = _evaluate(m, sc_n, q, q_tilde, lag, True)
        res = float(np.abs(g[m.free]).max())
        if res <= rtol * scale:
            return q, it
        p = np.zeros(3 * sc_n.Ns)
        p[free3] = -np.linalg.solve(H[np.ix_(free3, free3)], g.ravel()[free3])
        P = p.reshape(-1, 3)
        if np.abs(P).max() <= 4.0 * np.finfo(float).eps * np.abs(q).max():
            return q, it
        alpha = accd(sc_n, x, embed(sc_n, P, displacement=True))["alpha"]
        slope = float(g.ravel() @ p)
        while True:
            phi_t, g_t, _, _, _ = _evaluate(m, sc_n, q + alpha * P, q_tilde, lag, False)
            # Armijo, or (energy flat to rounding) a smaller residual
            if phi_t <= phi + 1e-4 * alpha * slope or (
                    phi_t - phi <= 1e-14 * abs(phi) and float(np.abs(g_t[m.free]).max()) < res):
                break
            alpha *= 0.5
            if alpha < 1e-20:
                return q, it          # no further progress at this precision
        q = q + alpha * P
    return q, max_iter


# ------------------------------------------------------------------ trajectory + adjoint
def initial_lag(m: Model, kappa: float):
    """Lagged friction state of the whole trajectory, taken once at its start."""
    if m.sc.params["mu"] == 0.0:
        return None
    sc0 = shifted_scene(m, np.zeros(3), kappa)
    x0 = embed(sc0, m.sc.q0)
    return friction_lag(sc0, x0, pairs(sc0, x0))


def trajectory(m: Model, theta: float, kappa: float, n_steps: Optional[int] = None):
    """States q_0 .. q_N for pad displacement theta per step and contact stiffness kappa."""
    N = m.sc.n_steps if n_steps is None else n_steps
    lag = initial_lag(m, kappa)
    every = getattr(m.sc, "lag_every_step", False) and m.sc.params["mu"] > 0
    pad_dir = np.asarray(getattr(m.sc, "pad_dir", (0.0, 0.0, 1.0)), float)
    presc = getattr(m.sc, "prescribed_q", None)
    qs = [m.sc.q0.copy()]
    prev2 = m.sc.q0.copy()
    iters = []
    for n in range(1, N + 1):
        if every and n > 1:
            scp = shifted_scene(m, (n - 1) * theta * pad_dir, kappa)
            xp = embed(scp, qs[-1])
            lag = friction_lag(scp, xp, pairs(scp, xp))
        q, it = newton_step(m, qs[-1], prev2, n * theta * pad_dir, kappa, lag,
                            q_fixed=None if presc is None else presc(n))
        prev2 = qs[-1]
        qs.append(q)
        iters.append(it)
    return qs, lag, iters


def loss(m: Model, q_N, theta: float, kappa: float, lag, N: int):
    """Sum of squared reduced contact forces at the final state."""
    sc_n = shifted_scene(m, N * theta * m.sc.pad_dir, kappa)
    _, _, r = contact(sc_n, q_N, lag)
    return float(np.sum(r["g"] ** 2)), r["g"]


def adjoint(m: Model, theta: float, kappa: float, n_steps: Optional[int] = None) -> Dict[str, float]:
    """dL/dtheta and dL/dkappa of L = ||g_c(q_N)||^2 by the discrete adjoint of the
    trajectory (implicit differentiation of every step's optimality condition
    F_n = M (q_n - 2 q_{n-1} + q_{n-2}) + h^2 (grad Phi - f + g_c(q_n)) = 0)."""
    N = m.sc.n_steps if n_steps is None else n_steps
    qs, lag, _ = trajectory(m, theta, kappa, N)
    h2 = m.h ** 2
    free3 = np.repeat(m.free, 3)
    kin = m.sc.kinematic
    ns = m.sc.Ns

    def kin_dir_u(n):
        u = np.zeros((m.sc.Nv, 3))
        u[kin] = n * m.sc.pad_dir
        return u

    L, gN = loss(m, qs[N], theta, kappa, lag, N)
    scN = shifted_scene(m, N * theta * m.sc.pad_dir, kappa)
    xN = embed(scN, qs[N])
    prsN = pairs(scN, xN)
    qbar = [np.zeros((ns, 3)) for _ in range(N + 1)]
    hv, _ = hvp(scN, xN, prsN, lag, embed(scN, gN, displacement=True))
    qbar[N] += 2.0 * hv
    hk, _ = hvp(scN, xN, prsN, lag, kin_dir_u(N))
    tbar = 2.0 * float(np.sum(gN * hk))
    kbar = 2.0 * float(np.sum(gN * gN)) / kappa
    for n in range(N, 0, -1):
        sc_n = shifted_scene(m, n * theta * m.sc.pad_dir, kappa)
        x, prs, r = contact(sc_n, qs[n], lag, project=False)
        A = np.kron(m.M, np.eye(3)) + h2 * (elastic_hessian(m, qs[n], False) + _blocks_to_dense(ns, r))
        z = np.zeros(3 * ns)
        z[free3] = np.linalg.solve(A[np.ix_(free3, free3)], qbar[n].ravel()[free3])
        Z = z.reshape(-1, 3)
        MZ = m.M @ Z
        if n - 1 >= 1:
            qbar[n - 1] += 2.0 * MZ
        if n - 2 >= 1:
            qbar[n - 2] -= MZ
        hk, _ = hvp(sc_n, x, prs, lag, kin_dir_u(n))
        tbar -= h2 * float(np.sum(Z * hk))
        kbar -= h2 * float(np.sum(Z * r["g"])) / kappa
    return dict(loss=L, dtheta=tbar, dkappa=kbar)
