"""Reduced Newton driver of Embedded IPC on one GPU: backward Euler on the cage
coordinates q (Sec. III-A), minimising the incremental potential

    E_IPC(q) = 1/2 (q - q~)^T M^q (q - q~) + h^2 (Phi(q) - f^q . q + B(Jq) + D(Jq)),
    q~ = q^n + h qdot^n,   M^q = J^T M J,   f^q = J^T f_ext          (Sec. III-A, III-B, III-D)

by Newton iterations whose step is capped by the CCD bound and then backtracked
(Sec. III-C).  The contact terms B, D and their derivatives come from the CUDA contact
stage (ContactScene); the cage elasticity Phi and the mass are torch operations on the
same device.  Two linear solvers:
  * dense (cage-sized systems): the exact Hessian wherever it is positive definite on the
    free DoFs (Cholesky test), the projected-Newton one otherwise;
  * PCG on the 3x3-block sparse matrices (surface-sized scenes): M + h^2 H_el assembled on
    the cage's tet-adjacency pattern, the contact H_r as the library returns it, products by
    the library's BSR SpMV, block-Jacobi preconditioning, the projected (SPD) Hessian.
Dirichlet nodes are either fixed at their start positions or follow a prescribed motion
(`prescribed_nodes`, `prescribed_q(n)` on the scene).  Materials are per body when the
scene gives `materials` (body id -> E, nu, rho), else one `material`.

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
from .elastic import CorotationalCage, FixedScatter, lame


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
        V = V + FixedScatter(t, sc.Nv)((vol / 3.0)[:, None].expand(-1, 3).reshape(-1))
    return V


@dataclass
class StepInfo:
    """How a Newton solve ended.  `reason` is "residual" (free residual below rtol times
    the largest force term), "step" (the Newton step fell below four ulps of the positions:
    the residual is at its rounding floor), "line_search" (backtracking found no decrease
    down to alpha < 1e-20) or "max_iter".  Only the first two are converged."""
    iterations: int
    residual: float
    exact_hessian_steps: int
    krylov_iterations: int = 0
    reason: str = "residual"

    @property
    def converged(self) -> bool:
        return self.reason in ("residual", "step")


class NewtonError(RuntimeError):
    """A Newton solve that stopped without converging (line search or iteration cap)."""

    def __init__(self, info: StepInfo):
        super().__init__(f"Newton step did not converge: {info.reason} after {info.iterations} iterations, "
                         f"relative residual {info.residual:.3e}")
        self.info = info


class Simulator:
    """Driver for one scene with `q0`, `gravity`, `fixed_nodes` (or `prescribed_nodes` and
    `prescribed_q`), and `material` (or per-body `materials`) attributes (see scenes)."""

    def __init__(self, scene, device: str = "cuda", solver: str = "auto", pair_capacity: int = 1 << 18,
                 bsr_capacity: int = 1 << 20, rec_capacity: int = 1 << 22, dense_limit: int = 12000):
        self.sc = scene
        self.dev = torch.device(device)
        self.cs = binding.ContactScene(scene, pair_capacity=pair_capacity, bsr_capacity=bsr_capacity,
                                       rec_capacity=rec_capacity, device=device)
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
        tet_of_np = np.array([row_of[tuple(r)] for r in np.asarray(scene.cage_idx)[emb_np].tolist()], np.int64)
        tet_of = torch.as_tensor(tet_of_np, device=self.dev)
        V_T = FixedScatter(tet_of, tets.shape[0])(Vk[emb])
        # materials: one, or one per body (a tet takes the body of the vertices inside it)
        T = tets.shape[0]
        body_np = np.asarray(scene.body)[emb_np]
        mats = getattr(scene, "materials", None)
        tet_body = np.zeros(T, np.int64)
        tet_body[tet_of_np] = body_np
        if mats:
            E = np.array([mats[int(b)]["E"] for b in tet_body]); nu = np.array([mats[int(b)]["nu"] for b in tet_body])
            rho_v = np.array([mats[int(b)]["rho"] for b in body_np])
        else:
            E = np.full(T, scene.material["E"]); nu = np.full(T, scene.material["nu"])
            rho_v = np.full(len(body_np), scene.material["rho"])
        mu, lam = lame(E, nu)
        self.elastic = CorotationalCage(tets, self.q0, V_T, torch.as_tensor(mu, **f64), torch.as_tensor(lam, **f64))
        # mass on the cage's block pattern (each vertex's four nodes belong to one tet)
        self.row_ptr, self.col, self.slot = self.elastic.block_pattern()
        self.nnzb = int(self.col.shape[0])
        m = torch.as_tensor(rho_v, **f64) * Vk[emb]
        ie, we = idx[emb], w[emb]
        vslot = self.slot[tet_of]                                       # [nv_emb,4,4]
        # the vertex's node order is its tet's node order (cage_idx row = tet row)
        Mb = FixedScatter(vslot, self.nnzb)((m[:, None, None] * we[:, :, None] * we[:, None, :]).reshape(-1))
        self.Mb = Mb
        eye = torch.eye(3, **f64)
        self.M_blocks = Mb[:, None, None] * eye
        rows = torch.repeat_interleave(torch.arange(self.Ns, device=self.dev),
                                       (self.row_ptr[1:] - self.row_ptr[:-1]).long())
        self.diag_slot = torch.nonzero(rows == self.col.long()).squeeze(1)   # one per row
        g = torch.as_tensor(np.asarray(scene.gravity, float), **f64)
        self.f_ext = FixedScatter(ie, self.Ns)(((m[:, None] * we).reshape(-1, 1)) * g[None, :])
        active = torch.zeros(self.Ns, dtype=torch.bool, device=self.dev)
        active[tets[V_T > 0].reshape(-1)] = True
        fixed = getattr(scene, "prescribed_nodes", None)
        if fixed is None:
            fixed = scene.fixed_nodes
        self.free = active & ~torch.as_tensor(fixed, device=self.dev)
        self.free3 = self.free.repeat_interleave(3)
        self.x_kin0 = torch.as_tensor(scene.x_kin, **f64)
        self.pad_dir = torch.as_tensor(np.asarray(getattr(scene, "pad_dir", (0.0, 0.0, 1.0)), float), **f64)
        self.kappa = float(scene.params["kappa"])
        n_free = int(self.free.sum()) * 3
        self.solver = ("dense" if n_free <= dense_limit else "pcg") if solver == "auto" else solver
        if self.solver == "dense":
            M = torch.zeros((self.Ns, self.Ns), **f64)
            r_i = rows
            M.index_put_((r_i, self.col.long()), Mb, accumulate=True)
            self.M = M
            # free-DoF numbering for the dense systems (-1 on Dirichlet DoFs)
            fi = torch.full((3 * self.Ns,), -1, dtype=torch.int64, device=self.dev)
            fi[self.free3] = torch.arange(int(self.free3.sum()), device=self.dev)
            self.free_index = fi
            self.M3f = torch.kron(M[self.free][:, self.free], eye).contiguous()
        self.pcg_rtol = 1e-10
        self.pcg_max = 5000

    # ---------------------------------------------------------------- linear algebra
    def _bsr_apply(self, row_ptr, col, val, x, alpha=1.0, beta=0.0, out=None):
        return binding.bsr_spmv(row_ptr, col, val.reshape(-1, 9), x.contiguous(), out=out, alpha=alpha, beta=beta)

    def mass_apply(self, X):
        """M^q X for X [Ns,3]."""
        return self._bsr_apply(self.row_ptr, self.col, self.M_blocks, X)

    # ---------------------------------------------------------------- contact terms
    def set_state(self, shift, kappa: float):
        """Kinematic vertices displaced by `shift` (3-vector) from their start; contact
        stiffness kappa."""
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

    def contact(self, q, lag, project: bool = True, hessian: bool = True, dense: bool = True):
        pairs = self.cs.build_candidates(q)
        E, g, H = self.cs.eval_contact(q, pairs, lag, project=project)
        if not hessian:
            return pairs, E, g, None
        return pairs, E, g, (self._bsr_dense(H) if dense else H)

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

    def _forces(self, q, q_tilde, lag):
        h2 = self.h ** 2
        pairs, E, gc, _ = self.contact(q, lag, project=True, hessian=False)
        d = q - q_tilde
        Md = self.mass_apply(d)
        ge = self.elastic.gradient(q)
        phi = 0.5 * (d * Md).sum() + h2 * (self.elastic.energy(q) - (self.f_ext * q).sum() + E[0])
        g = Md + h2 * (ge - self.f_ext + gc)
        scale = (Md.abs() + h2 * (ge.abs() + self.f_ext.abs() + gc.abs()))[self.free].max()
        return float(phi), g, float(scale)

    # ---------------------------------------------------------------- Newton directions
    def _free_block(self, rows, cols, vals, out):
        """Accumulate dense entries (DoF rows, cols, values) into the free-DoF block."""
        fr, fc = self.free_index[rows], self.free_index[cols]
        keep = (fr >= 0) & (fc >= 0)
        out.index_put_((fr[keep], fc[keep]), vals[keep], accumulate=True)

    def _system_dense(self, q, lag, project: bool):
        """M + h^2 (hess Phi + H_c) on the free DoFs (exact, or projected)."""
        h2 = self.h ** 2
        A = self.M3f.clone()
        Ht = h2 * self.elastic.tet_hessians(q, project)
        T = Ht.shape[0]
        d = self.elastic.dofs
        self._free_block(d[:, :, None].expand(T, 12, 12).reshape(-1), d[:, None, :].expand(T, 12, 12).reshape(-1),
                         Ht.reshape(-1), A)
        _, _, _, Hc = self.contact(q, lag, project=project, dense=False)
        nnzb = int(Hc.nnzb.item())
        rp = Hc.row_ptr.long()
        rows = torch.repeat_interleave(torch.arange(self.Ns, device=self.dev), rp[1:] - rp[:-1])
        cols = Hc.col[:nnzb].long()
        ar = torch.arange(3, device=self.dev)
        r3 = (3 * rows[:, None, None] + ar[None, :, None]).expand(nnzb, 3, 3).reshape(-1)
        c3 = (3 * cols[:, None, None] + ar[None, None, :]).expand(nnzb, 3, 3).reshape(-1)
        self._free_block(r3, c3, h2 * Hc.val[:nnzb].reshape(-1), A)
        return A

    def _direction_dense(self, q, lag, g):
        A = self._system_dense(q, lag, project=False)
        L, info = torch.linalg.cholesky_ex(A)
        exact = int(info.item()) == 0
        if not exact:
            A = self._system_dense(q, lag, project=True)
            L, info = torch.linalg.cholesky_ex(A)
            if int(info.item()) != 0:          # semidefinite at rounding: a dense LU instead
                L = None
        b = -g.reshape(-1)[self.free3]
        x = torch.cholesky_solve(b[:, None], L).squeeze(1) if L is not None else torch.linalg.solve(A, b)
        p = torch.zeros(3 * self.Ns, dtype=torch.float64, device=self.dev)
        p[self.free3] = x
        return p.reshape(-1, 3), exact, 0

    def _direction_pcg(self, q, lag, g):
        """A p = -g on the free DoFs with A = M + h^2 (P+ hess Phi + H_c+) by block-Jacobi PCG."""
        h2 = self.h ** 2
        _, _, _, Hc = self.contact(q, lag, project=True, dense=False)
        Ael = self.M_blocks + h2 * self.elastic.assemble_blocks(self.elastic.tet_hessians(q, True), self.slot, self.nnzb)
        nnzb_c = int(Hc.nnzb.item())
        mask = self.free[:, None].to(torch.float64)
        # block-Jacobi: diagonal blocks of both matrices
        D = Ael[self.diag_slot].clone()
        rp = Hc.row_ptr.long()
        rows_c = torch.repeat_interleave(torch.arange(self.Ns, device=self.dev), rp[1:] - rp[:-1])
        on_diag = torch.nonzero(rows_c == Hc.col[:nnzb_c].long()).squeeze(1)
        D = D + FixedScatter(rows_c[on_diag], self.Ns)(h2 * Hc.val[on_diag].reshape(-1, 3, 3))
        eye = torch.eye(3, dtype=torch.float64, device=self.dev)
        D = torch.where(self.free[:, None, None], D, eye)
        Dinv = torch.linalg.inv(D)
        tmp = torch.empty((self.Ns, 3), dtype=torch.float64, device=self.dev)

        def apply(X):
            X = (X * mask).contiguous()
            Y = self._bsr_apply(self.row_ptr, self.col, Ael, X)
            self._bsr_apply(Hc.row_ptr, Hc.col, Hc.val[:nnzb_c], X, alpha=h2, beta=1.0, out=Y)
            return Y * mask

        b = -(g * mask)
        x = torch.zeros_like(b)
        r = b.clone()
        z = torch.einsum("nij,nj->ni", Dinv, r) * mask
        p = z.clone()
        rz = (r * z).sum()
        b_norm = float(torch.linalg.norm(b))
        it = 0
        if b_norm == 0.0:
            return x, False, 0
        for it in range(1, self.pcg_max + 1):
            Ap = apply(p)
            alpha = rz / (p * Ap).sum()
            x = x + alpha * p
            r = r - alpha * Ap
            if it % 10 == 0 and float(torch.linalg.norm(r)) <= self.pcg_rtol * b_norm:
                break
            z = torch.einsum("nij,nj->ni", Dinv, r) * mask
            rz_new = (r * z).sum()
            p = z + (rz_new / rz) * p
            rz = rz_new
        return x, False, it

    # ---------------------------------------------------------------- one time step
    def step(self, q_prev, q_prev2, shift, kappa: float, lag, rtol: float = 1e-12, max_iter: int = 100,
             q_fixed=None, strict: bool = True):
        """q^{n+1} with the kinematic vertices at `shift` and the Dirichlet nodes at q_fixed
        (their start positions if None): Newton with the CCD step bound and backtracking
        until the free residual is below rtol times the largest force term, or the step is
        below four ulps of the positions.  The returned StepInfo says which; a solve that
        ends otherwise (backtracking exhausted, iteration cap) raises NewtonError when
        `strict`, else comes back with that reason."""
        self.set_state(shift, kappa)
        q_tilde = 2.0 * q_prev - q_prev2
        q = q_prev.clone()
        if q_fixed is not None:
            q = torch.where(self.free[:, None], q, q_fixed)
        n_exact = 0
        n_kry = 0
        eps = float(np.finfo(np.float64).eps)
        res = float("inf")
        scale = 1.0
        for it in range(max_iter):
            phi, g, scale = self._forces(q, q_tilde, lag)
            res = float(g[self.free].abs().max())
            if res <= rtol * scale:
                return q, StepInfo(it, res / scale, n_exact, n_kry, "residual")
            if self.solver == "dense":
                P, exact, k = self._direction_dense(q, lag, g)
            else:
                P, exact, k = self._direction_pcg(q, lag, g)
            n_exact += int(exact)
            n_kry += k
            if float(P.abs().max()) <= 4.0 * eps * float(q.abs().max()):
                return q, StepInfo(it, res / scale, n_exact, n_kry, "step")
            x = self.cs.embed(q)
            dx = self.cs.embed(P, displacement=True)
            alpha = float(self.cs.accd_toi(x, dx).item())
            slope = float((g * P).sum())
            while True:
                phi_t, g_t, _ = self._forces(q + alpha * P, q_tilde, lag)
                if phi_t <= phi + 1e-4 * alpha * slope or (
                        phi_t - phi <= 1e-14 * abs(phi) and float(g_t[self.free].abs().max()) < res):
                    break
                alpha *= 0.5
                if alpha < 1e-20:
                    return q, self._stalled(StepInfo(it, res / scale, n_exact, n_kry, "line_search"), strict)
            q = q + alpha * P
        return q, self._stalled(StepInfo(max_iter, res / scale, n_exact, n_kry, "max_iter"), strict)

    @staticmethod
    def _stalled(info: StepInfo, strict: bool) -> StepInfo:
        if strict:
            raise NewtonError(info)
        return info

    def prescribed(self, n: int):
        """Positions of the Dirichlet nodes at step n (None: their start positions)."""
        f = getattr(self.sc, "prescribed_q", None)
        if f is None:
            return None
        return torch.as_tensor(f(n), dtype=torch.float64, device=self.dev)

    def trajectory(self, theta: float = 0.0, kappa: Optional[float] = None, n_steps: Optional[int] = None,
                   rtol: float = 1e-12):
        kappa = self.kappa if kappa is None else float(kappa)
        N = self.sc.n_steps if n_steps is None else int(n_steps)
        lag = self.initial_lag(kappa)
        every = getattr(self.sc, "lag_every_step", False) and self.sc.params["mu"] > 0
        qs = [self.q0.clone()]
        prev2 = self.q0.clone()
        infos = []
        for n in range(1, N + 1):
            if every and n > 1:
                self.set_state((n - 1) * theta * self.pad_dir, kappa)
                lag = self.cs.friction_lag(qs[-1], self.cs.build_candidates(qs[-1], out=self.cs.new_pairs()))
            q, info = self.step(qs[-1], prev2, n * theta * self.pad_dir, kappa, lag, rtol=rtol, q_fixed=self.prescribed(n))
            prev2 = qs[-1]
            qs.append(q)
            infos.append(info)
        return qs, lag, infos

    def contact_force(self, q, shift, kappa: float, lag):
        """Reduced contact gradient g_c at q with the kinematic vertices at `shift`."""
        self.set_state(shift, kappa)
        _, _, g, _ = self.contact(q, lag, hessian=False)
        return g
