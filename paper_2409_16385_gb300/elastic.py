"""Cage elasticity of Embedded IPC on the GPU (torch): Phi(q) = sum_T V_T Psi(F_T) with the
linear corotational density Psi(F) = mu ||F - R||^2 + lambda/2 (tr S - 3)^2, F = R S the
polar decomposition, F_T = D_T (D_T^0)^{-1}, and V_T the sum of the per-vertex volumes of
the embedded vertices inside tet T (Sec. III-D; the material of Sec. IV-A).

Derivatives are closed form.  P = dPsi/dF = 2 mu (F - R) + lambda (tr S - 3) R.  For the
exact Hessian, the rotation's differential is dR = R [w]_x with
(tr(S) I - S) w = axial(R^T dF - dF^T R), because R^T dF - dF^T R = W S + S W for the
skew W = R^T dR; and d tr S = R : dF.  Hence
    dP = 2 mu (dF - dR) + lambda (R : dF) R + lambda (tr S - 3) dR.
The projected-Newton Hessian clamps the negative eigenvalues of each tet's 9 x 9
Hessian in F.
"""
from __future__ import annotations

import torch


class FixedScatter:
    """out[idx[k]] += v[k] in an order that depends only on idx: every target's
    contributions, in increasing k, are gathered into one row of an [n, width] table
    (padded with a zero entry) and summed along the row by a fixed-shape reduction.
    torch's index_add_ on CUDA adds with atomics, whose order (and so the rounding of the
    result) changes from run to run; this form gives the same bits on every run."""

    def __init__(self, idx, n: int):
        idx = idx.reshape(-1).long()
        self.n, self.m = int(n), int(idx.numel())
        dev = idx.device
        counts = torch.bincount(idx, minlength=self.n)
        width = max(int(counts.max()) if self.m else 0, 1)
        order = torch.argsort(idx, stable=True)
        start = torch.cumsum(counts, 0) - counts
        rank = torch.arange(self.m, device=dev) - start[idx[order]]
        table = torch.full((self.n, width), self.m, dtype=torch.int64, device=dev)
        table[idx[order], rank] = order
        self.table = table

    def __call__(self, v):
        tail = v.shape[1:]
        flat = v.reshape(self.m, -1)
        padded = torch.cat([flat, torch.zeros((1, flat.shape[1]), dtype=v.dtype, device=v.device)])
        return padded[self.table].sum(1).reshape((self.n,) + tuple(tail))


def lame(E: float, nu: float):
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def _skew(w):
    z = torch.zeros_like(w[..., 0])
    return torch.stack([torch.stack([z, -w[..., 2], w[..., 1]], -1),
                        torch.stack([w[..., 2], z, -w[..., 0]], -1),
                        torch.stack([-w[..., 1], w[..., 0], z], -1)], -2)


def _axial(K):
    return torch.stack([K[..., 2, 1], K[..., 0, 2], K[..., 1, 0]], -1)


class CorotationalCage:
    """Elasticity of one cage: tets [T,4] (node ids), rest positions q0 [Ns,3], tet
    volumes V_T [T] (device tensors, float64); Lame parameters mu, lam as numbers or as
    per-tet tensors [T] (several bodies with their own materials)."""

    def __init__(self, tets, q0, V_T, mu, lam):
        self.tets = tets.long()
        self.ns = q0.shape[0]
        T = self.tets.shape[0]
        as_t = lambda a: (a.to(q0) if torch.is_tensor(a) else torch.full((T,), float(a), dtype=q0.dtype,
                                                                          device=q0.device))
        self.mu, self.lam = as_t(mu), as_t(lam)
        Dm = self._ds(q0)
        self.Dm_inv = torch.linalg.inv(Dm)
        self.V_T = V_T
        # B maps a tet's 12 node displacements (node-major 3a + c) to dF (row-major 3i + j)
        T = self.tets.shape[0]
        B = torch.zeros((T, 9, 12), dtype=q0.dtype, device=q0.device)
        colsum = self.Dm_inv.sum(1)                     # sum_k Dminv[k, j]
        for i in range(3):
            for j in range(3):
                B[:, 3 * i + j, i] = -colsum[:, j]      # node 0, component i
                for a in range(1, 4):
                    B[:, 3 * i + j, 3 * a + i] = self.Dm_inv[:, a - 1, j]
        self.B = B
        self.dofs = (3 * self.tets[:, :, None] + torch.arange(3, device=q0.device)[None, None, :]).reshape(T, 12)
        # node of each (tet, local node) entry, for the deterministic nodal scatter
        self._node_scatter = FixedScatter(self.tets, self.ns)
        self._block_scatter = None

    def _ds(self, q):
        t = self.tets
        return torch.stack([q[t[:, 1]] - q[t[:, 0]], q[t[:, 2]] - q[t[:, 0]], q[t[:, 3]] - q[t[:, 0]]], dim=2)

    def deformation(self, q):
        return self._ds(q) @ self.Dm_inv

    @staticmethod
    def polar(F):
        U, s, Vh = torch.linalg.svd(F)
        flip = (torch.linalg.det(U) * torch.linalg.det(Vh)) < 0
        if bool(flip.any()):
            U = U.clone(); s = s.clone()
            U[flip, :, 2] = -U[flip, :, 2]
            s[flip, 2] = -s[flip, 2]
        R = U @ Vh
        S = Vh.transpose(-1, -2) @ torch.diag_embed(s) @ Vh
        return R, 0.5 * (S + S.transpose(-1, -2))

    def _stress(self, F):
        R, S = self.polar(F)
        tr = S.diagonal(dim1=-2, dim2=-1).sum(-1)
        P = 2.0 * self.mu[:, None, None] * (F - R) + (self.lam * (tr - 3.0))[:, None, None] * R
        return P, R, S, tr

    def _scatter(self, G):
        """dE/dDs per tet [T,3,3] (columns = nodes 1..3) -> nodal vectors [Ns,3]."""
        per_node = torch.cat([-G.sum(2)[:, None, :], G.transpose(1, 2)], dim=1)   # [T,4,3]
        return self._node_scatter(per_node.reshape(-1, 3))

    def energy(self, q) -> torch.Tensor:
        F = self.deformation(q)
        R, S = self.polar(F)
        tr = S.diagonal(dim1=-2, dim2=-1).sum(-1)
        D = F - R
        psi = self.mu * (D * D).sum((-1, -2)) + 0.5 * self.lam * (tr - 3.0) ** 2
        return (self.V_T * psi).sum()

    def gradient(self, q):
        P, _, _, _ = self._stress(self.deformation(q))
        return self._scatter(self.V_T[:, None, None] * (P @ self.Dm_inv.transpose(1, 2)))

    def _dP(self, dF, R, S, tr):
        trI = tr[:, None, None] * torch.eye(3, dtype=S.dtype, device=S.device) - S
        Rt = R.transpose(-1, -2)
        k = _axial(Rt @ dF - dF.transpose(-1, -2) @ R)
        w = torch.linalg.solve(trI, k.unsqueeze(-1)).squeeze(-1)
        dR = R @ _skew(w)
        RdF = (R * dF).sum((-1, -2))
        mu, lam = self.mu[:, None, None], self.lam[:, None, None]
        return 2.0 * mu * (dF - dR) + lam * RdF[:, None, None] * R + lam * (tr - 3.0)[:, None, None] * dR

    def hvp(self, q, v):
        """Exact Hessian of Phi at q times v [Ns,3]."""
        F = self.deformation(q)
        _, R, S, tr = self._stress(F)
        dF = self._ds(v) @ self.Dm_inv
        dP = self._dP(dF, R, S, tr)
        return self._scatter(self.V_T[:, None, None] * (dP @ self.Dm_inv.transpose(1, 2)))

    def tet_hessians(self, q, project: bool):
        """12 x 12 Hessian of V_T Psi per tet (node-major), exact or PSD-projected in F."""
        F = self.deformation(q)
        _, R, S, tr = self._stress(F)
        T = F.shape[0]
        E = torch.eye(9, dtype=F.dtype, device=F.device).reshape(9, 3, 3)
        cols = [self._dP(E[c].expand(T, 3, 3), R, S, tr).reshape(T, 9) for c in range(9)]
        HF = torch.stack(cols, dim=2)
        HF = 0.5 * (HF + HF.transpose(1, 2))
        if project:
            lam, V = torch.linalg.eigh(HF)
            HF = V @ torch.diag_embed(lam.clamp_min(0.0)) @ V.transpose(1, 2)
        return self.V_T[:, None, None] * (self.B.transpose(1, 2) @ HF @ self.B)

    def block_pattern(self):
        """3x3-block CSR pattern of the cage Hessian (node pairs sharing a tet) and, per tet,
        the block index of each (a, b) node pair: (row_ptr [Ns+1] int32, col int32,
        slot [T,4,4] int64)."""
        t = self.tets
        T = t.shape[0]
        I = t[:, :, None].expand(T, 4, 4).reshape(-1)
        J = t[:, None, :].expand(T, 4, 4).reshape(-1)
        key = I * self.ns + J
        uniq, inv = torch.unique(key, sorted=True, return_inverse=True)
        rows = uniq // self.ns
        counts = torch.bincount(rows, minlength=self.ns)
        row_ptr = torch.zeros(self.ns + 1, dtype=torch.int64, device=t.device)
        row_ptr[1:] = torch.cumsum(counts, 0)
        return row_ptr.to(torch.int32), (uniq % self.ns).to(torch.int32), inv.reshape(T, 4, 4)

    def assemble_blocks(self, Ht, slot, nnzb):
        """Per-tet 12 x 12 Hessians -> values [nnzb,3,3] on the block pattern."""
        T = Ht.shape[0]
        blocks = Ht.reshape(T, 4, 3, 4, 3).permute(0, 1, 3, 2, 4).reshape(T * 16, 3, 3)
        if self._block_scatter is None or self._block_scatter.n != nnzb:
            self._block_scatter = FixedScatter(slot, nnzb)
        return self._block_scatter(blocks)

    def assemble_dense(self, Ht):
        n = 3 * self.ns
        H = torch.zeros((n, n), dtype=Ht.dtype, device=Ht.device)
        T = Ht.shape[0]
        rows = self.dofs[:, :, None].expand(T, 12, 12).reshape(-1)
        cols = self.dofs[:, None, :].expand(T, 12, 12).reshape(-1)
        H.index_put_((rows, cols), Ht.reshape(-1), accumulate=True)
        return H
