"""Reduced Newton driver of Embedded IPC on one GPU: backward Euler on the cage
coordinates q (Sec. III-A), minimising the incremental potential

    E_IPC(q) = 1/2 (q - q~)^T M^q (q - q~) + h^2 (Phi(q) - f^q . q + B(Jq) + D(Jq)),
    q~ = q^n + h qdot^n,   M^q = J^T M J,   f^q = J^T f_ext          (Sec. III-A, III-B, III-D)

by Newton iterations whose step is capped by the CCD bound and then backtracked
(Sec. III-C).  The contact terms B, D and their derivatives come from the CUDA contact
stage (ContactScene); the cage elasticity Phi, the mass and the linear solves run as
torch operations on the same device.  The Newton Hessian is the exact one wherever it is
positive definite on the free DoFs (tested by Cholesky) and the projected-Newton one
otherwise.  Systems are small and dense here (the cage DoFs, not the surface).

Per-vertex volumes V_k of an embedded closed surface are the cones of its triangles to
the body's centroid, a third to each vertex; V_T sums V_k over the vertices embedded in T,
and the lumped full-space mass is rho V_k (Sec. III-D).  External force: gravity, with the
potential E_ext = -f^q . q.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import binding
from .elastic import CorotationalCage, lame


def _vertex_volumes(sc, x) -> torch.Tensor:
    dev = x.device
    V = torch.zeros(sc.Nv, dtype=torch.float64, device=dev)
    kin = torch.as_tensor(sc.kinematic, device=dev)
    body = torch.as_tensor(sc.body, device=dev)
    tris = torch.as_tensor(sc.tris, device=dev).long()
    for b in torch.unique(body).tolist():
        members = body == b
        if bool(kin[members].all()):
            continue
        t = tris[members[tris[:, 0]]]
        c = x[members].mean(0)
        a0, a1, a2 = x[t[:, 0]] - c, x[t[:, 1]] - c, x[t[:, 2]] - c
        vol = (a0 * torch.linalg.cross(a1, a2)).sum(1) / 6.0
        if float(vol.sum()) < 0:
            vol = -vol
        for k in range(3):
            V.index_add_(0, t[:, k], vol / 3.0)
    return V


@dataclass
class StepInfo:
    iterations: int
    residual: float
    exact_hessian_steps: int


class Simulator:
    """Driver for one scene with `material`, `gravity`, `fixed_nodes`, `q0` attributes
    (see scenes.pad_lift)."""

    def __init__(self, scene, device: str = "cuda", pair_capacity: int = 1 << 18, bsr_capacity: int = 1 << 20):
        self.sc = scene
        self.dev = torch.device(device)
        self.cs = binding.ContactScene(scene, pair_capacity=pair_capacity, bsr_capacity=bsr_capacity,
                                       rec_capacity=1 << 22, device=device)
        f64 = dict(dtype=torch.float64, device=self.dev)
        self.h = float(scene.params["h"])
        self.q0 = torch.as_tensor(scene.q0, **f64)
        self.Ns = scene.Ns
        idx = torch.as_tensor(scene.cage_idx, device=self.dev).long()
        w = torch.as_tensor(scene.w, **f64)
        emb = ~torch.as_tensor(scene.kinematic, device=self.dev)
        self.kin = ~emb
        x0 = self.cs.embed(self.q0)
        Vk = _vertex_volumes(scene, x0) * emb
        # tet of each embedded vertex: its cage_idx row is that tet's node list (set-up only)
        tets = torch.as_tensor(scene.cage_tets, device=self.dev).long()
        row_of = {tuple(r): i for i, r in enumerate(np.asarray(scene.cage_tets).tolist())}
        emb_np = ~np.asarray(scene.kinematic)
        tet_of = torch.as_tensor([row_of[tuple(r)] for r in np.asarray(scene.cage_idx)[emb_np].tolist()],
                                 device=self.dev)
        V_T = torch.zeros(tets.shape[0], **f64).index_add_(0, tet_of, Vk[emb])
        mu, lam = lame(scene.material["E"], scene.material["nu"])
        self.elastic = CorotationalCage(tets, self.q0, V_T, mu, lam)
        rho = float(scene.material["rho"])
        m = rho * Vk[emb]
        ie, we = idx[emb], w[emb]
        M = torch.zeros((self.Ns, self.Ns), **f64)
        M.index_put_((ie[:, :, None].expand(-1, 4, 4).reshape(-1), ie[:, None, :].expand(-1, 4, 4).reshape(-1)),
                     (m[:, None, None] * we[:, :, None] * we[:, None, :]).reshape(-1), accumulate=True)
        self.M = M
        self.M3 = torch.kron(M, torch.eye(3, **f64))
        g = torch.as_tensor(np.asarray(scene.gravity, float), **f64)
        f = torch.zeros((self.Ns, 3), **f64)
        f.index_add_(0, ie.reshape(-1), ((m[:, None] * we).reshape(-1, 1)) * g[None, :])
        self.f_ext = f
        active = torch.zeros(self.Ns, dtype=torch.bool, device=self.dev)
        active[tets[V_T > 0].reshape(-1)] = True
        self.free = active & ~torch.as_tensor(scene.fixed_nodes, device=self.dev)
        self.free3 = self.free.repeat_interleave(3)
        self.x_kin0 = torch.as_tensor(scene.x_kin, **f64)
        self.pad_dir = torch.as_tensor(np.asarray(scene.pad_dir, float), **f64)
        self.kappa = float(scene.params["kappa"])

    # ---------------------------------------------------------------- contact terms
    def set_state(self, shift, kappa: float):
        """Pad displaced by `shift` (3-vector) from its start; contact stiffness kappa."""
        self.cs.set_params(kappa=kappa)
        xk = self.x_kin0 + torch.where(self.kin[:, None], shift[None, :], torch.zeros_like(self.x_kin0))
        self.cs.set_kinematic(xk)

    def initial_lag(self, kappa: float):
        """Lagged friction state of a trajectory, taken once at its start."""
        if self.sc.params["mu"] == 0.0:
            return None
        self.set_state(torch.zeros(3, dtype=torch.float64, device=self.dev), kappa)
        pairs = self.cs.build_candidates(self.q0, out=self.cs.new_pairs())
        return self.cs.friction_lag(self.q0, pairs)

    def contact(self, q, lag, project: bool = True, hessian: bool = True):
        pairs = self.cs.build_candidates(q)
        E, g, H = self.cs.eval_contact(q, pairs, lag, project=project)
        Hd = self._bsr_dense(H) if hessian else None
        return pairs, E, g, Hd

    def _bsr_dense(self, H):
        n = 3 * self.Ns
        nnzb = int(H.nnzb.item())
        rp = H.row_ptr.long()
        rows = torch.repeat_interleave(torch.arange(self.Ns, device=self.dev), rp[1:] - rp[:-1])
        cols = H.col[:nnzb].long()
        r3 = (3 * rows[:, None, None] + torch.arange(3, device=self.dev)[None, :, None]).expand(nnzb, 3, 3)
        c3 = (3 * cols[:, None, None] + torch.arange(3, device=self.dev)[None, None, :]).expand(nnzb, 3, 3)
        D = torch.zeros((n, n), dtype=torch.float64, device=self.dev)
        D.index_put_((r3.reshape(-1), c3.reshape(-1)), H.val[:nnzb].reshape(-1), accumulate=True)
        return D

    def _evaluate(self, q, q_tilde, lag, hessian: bool):
        h2 = self.h ** 2
        pairs, E, gc, _ = self.contact(q, lag, project=True, hessian=False)
        d = q - q_tilde
        Md = self.M @ d
        ge = self.elastic.gradient(q)
        phi = 0.5 * (d * Md).sum() + h2 * (self.elastic.energy(q) - (self.f_ext * q).sum() + E[0])
        g = Md + h2 * (ge - self.f_ext + gc)
        scale = (Md.abs() + h2 * (ge.abs() + self.f_ext.abs() + gc.abs()))[self.free].max()
        H = None
        exact = False
        if hessian:
            _, _, _, Hc = self.contact(q, lag, project=False)
            H = self.M3 + h2 * (self.elastic.assemble_dense(self.elastic.tet_hessians(q, False)) + Hc)
            Hf = H[self.free3][:, self.free3]
            _, info = torch.linalg.cholesky_ex(Hf)
            exact = int(info.item()) == 0
            if not exact:
                _, _, _, Hcp = self.contact(q, lag, project=True)
                H = self.M3 + h2 * (self.elastic.assemble_dense(self.elastic.tet_hessians(q, True)) + Hcp)
        return float(phi), g, float(scale), H, exact

    # ---------------------------------------------------------------- one time step
    def step(self, q_prev, q_prev2, shift, kappa: float, lag, rtol: float = 1e-12, max_iter: int = 100):
        """q^{n+1} for the pad at `shift`: Newton with the CCD step bound and backtracking
        until the free residual is below rtol times the largest force term, or the step is
        below four ulps of the positions."""
        self.set_state(shift, kappa)
        q_tilde = 2.0 * q_prev - q_prev2
        q = q_prev.clone()
        n_exact = 0
        eps = float(np.finfo(np.float64).eps)
        for it in range(max_iter):
            phi, g, scale, H, exact = self._evaluate(q, q_tilde, lag, True)
            n_exact += int(exact)
            res = float(g[self.free].abs().max())
            if res <= rtol * scale:
                return q, StepInfo(it, res / scale, n_exact)
            p = torch.zeros(3 * self.Ns, dtype=torch.float64, device=self.dev)
            p[self.free3] = -torch.linalg.solve(H[self.free3][:, self.free3], g.reshape(-1)[self.free3])
            P = p.reshape(-1, 3)
            if float(P.abs().max()) <= 4.0 * eps * float(q.abs().max()):
                return q, StepInfo(it, res / scale, n_exact)
            x = self.cs.embed(q)
            dx = self.cs.embed(P, displacement=True)
            alpha = float(self.cs.accd_toi(x, dx).item())
            slope = float((g.reshape(-1) * p).sum())
            while True:
                phi_t, g_t, _, _, _ = self._evaluate(q + alpha * P, q_tilde, lag, False)
                if phi_t <= phi + 1e-4 * alpha * slope or (
                        phi_t - phi <= 1e-14 * abs(phi) and float(g_t[self.free].abs().max()) < res):
                    break
                alpha *= 0.5
                if alpha < 1e-20:
                    return q, StepInfo(it, res / scale, n_exact)
            q = q + alpha * P
        return q, StepInfo(max_iter, res / scale, n_exact)

    def trajectory(self, theta: float, kappa: Optional[float] = None, n_steps: Optional[int] = None):
        kappa = self.kappa if kappa is None else float(kappa)
        N = self.sc.n_steps if n_steps is None else int(n_steps)
        lag = self.initial_lag(kappa)
        qs = [self.q0.clone()]
        prev2 = self.q0.clone()
        infos = []
        for n in range(1, N + 1):
            q, info = self.step(qs[-1], prev2, n * theta * self.pad_dir, kappa, lag)
            prev2 = qs[-1]
            qs.append(q)
            infos.append(info)
        return qs, lag, infos

    def contact_force(self, q, shift, kappa: float, lag):
        """Reduced contact gradient g_c at q with the pad at `shift`."""
        self.set_state(shift, kappa)
        _, _, g, _ = self.contact(q, lag, hessian=False)
        return g
