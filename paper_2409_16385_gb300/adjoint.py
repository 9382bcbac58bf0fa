"""Differentiating through the contact stage and through whole trajectories.

`ContactForce` wraps the reduced contact gradient g_c(q; theta, kappa) of the CUDA library
as a torch.autograd.Function.  Its backward is one call of the Hessian-vector-product
kernel (eipc_contact_hvp) with the EXACT (unprojected) contact Hessian H:
    d/dq <G, g_c> = H_r G,
    d/dtheta <G, g_c> = n d . sum_kin (H J G)          (the pad at n theta d; H symmetric)
    d/dkappa <G, g_c> = <G, g_c> / kappa                (barrier and lagged friction are
                                                         both proportional to kappa)

`ImplicitStep` wraps one backward-Euler step q_n = argmin E_IPC (sim.Simulator.step) and
differentiates it implicitly: with F_n = M (q_n - 2 q_{n-1} + q_{n-2}) + h^2 (grad Phi -
f + g_c) = 0 on the free DoFs and A_n = dF_n/dq_n = M + h^2 (hess Phi + H_c) (exact),
a cotangent qbar gives z = A_n^{-1} qbar and
    qbar_{n-1} = 2 M z,   qbar_{n-2} = -M z,
    thetabar = -h^2 n d . sum_kin (H_c J z),   kappabar = -h^2 <z, g_c(q_n)> / kappa.
A_n z = qbar is solved densely (default) or matrix-free by MINRES on the HVPs of the
contact kernel and of the elasticity.

`trajectory_loss` chains the steps with activation checkpointing every k steps
(torch.utils.checkpoint), so the backward pass recomputes each segment's states from
its checkpoint instead of keeping all of them.  The friction lag state is taken once at
the trajectory's start; it is proportional to kappa and independent of theta.
"""
from __future__ import annotations

from typing import Optional

import torch
from torch.utils.checkpoint import checkpoint


class ContactForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, theta, kappa, sim, lag, n: int):
        shift = n * theta.detach() * sim.pad_dir
        g = sim.contact_force(q.detach(), shift, float(kappa.detach()), lag)
        ctx.sim, ctx.lag, ctx.n = sim, lag, n
        ctx.save_for_backward(q.detach(), theta.detach(), kappa.detach(), g)
        return g

    @staticmethod
    def backward(ctx, G):
        q, theta, kappa, g = ctx.saved_tensors
        sim, lag, n = ctx.sim, ctx.lag, ctx.n
        sim.set_state(n * theta * sim.pad_dir, float(kappa))
        pairs = sim.cs.build_candidates(q)
        Hg, kin = sim.cs.contact_hvp(q, pairs, G.contiguous(), lag=lag)
        d_theta = n * (kin * sim.pad_dir).sum()
        d_kappa = (G * g).sum() / kappa
        return Hg, d_theta, d_kappa, None, None, None


def _minres(apply, b, rtol: float = 1e-13, max_iter: int = 20000):
    """Paige-Saunders MINRES for a symmetric (possibly indefinite) operator."""
    x = torch.zeros_like(b)
    r = b.clone()
    beta = torch.linalg.norm(r)
    if float(beta) == 0.0:
        return x
    v_old = torch.zeros_like(b)
    v = r / beta
    c_old, s_old, c, s = 1.0, 0.0, 1.0, 0.0
    w_old = torch.zeros_like(b)
    w = torch.zeros_like(b)
    eta = float(beta)
    beta_k = float(beta)
    b_norm = float(beta)
    for _ in range(max_iter):
        Av = apply(v)
        alpha = float((v * Av).sum())
        u = Av - alpha * v - beta_k * v_old
        beta_next = float(torch.linalg.norm(u))
        delta = c * alpha - c_old * s * beta_k
        rho1 = (delta ** 2 + beta_next ** 2) ** 0.5
        rho2 = s * alpha + c_old * c * beta_k
        rho3 = s_old * beta_k
        c_new, s_new = delta / rho1, beta_next / rho1
        w_new = (v - rho3 * w_old - rho2 * w) / rho1
        x = x + c_new * eta * w_new
        eta = -s_new * eta
        if abs(eta) <= rtol * b_norm or beta_next == 0.0:
            break
        v_old, v = v, u / beta_next
        w_old, w = w, w_new
        c_old, s_old, c, s = c, s, c_new, s_new
        beta_k = beta_next
    return x


def _system(sim, q, theta, kappa, lag, n):
    sim.set_state(n * theta * sim.pad_dir, float(kappa))
    return sim.cs.build_candidates(q)


def solve_adjoint(sim, q, theta, kappa, lag, n, rhs, method: str = "dense"):
    """z with A_n z = rhs on the free DoFs (zero on the fixed ones)."""
    h2 = sim.h ** 2
    free3 = sim.free3
    z = torch.zeros_like(rhs).reshape(-1)
    if method == "dense":
        sim.set_state(n * theta * sim.pad_dir, float(kappa))
        A = sim._system_dense(q, lag, project=False)
        z[free3] = torch.linalg.solve(A, rhs.reshape(-1)[free3])
        return z.reshape(-1, 3)
    pairs = _system(sim, q, theta, kappa, lag, n)
    mask = sim.free[:, None].to(rhs.dtype)

    def apply(v):
        V = v.reshape(-1, 3) * mask
        Hc, _ = sim.cs.contact_hvp(q, pairs, V.contiguous(), lag=lag)
        out = sim.mass_apply(V) + h2 * (sim.elastic.hvp(q, V) + Hc)
        return (out * mask).reshape(-1)

    return _minres(apply, (rhs * mask).reshape(-1)).reshape(-1, 3)


class ImplicitStep(torch.autograd.Function):
    solver = "dense"

    @staticmethod
    def forward(ctx, q_prev, q_prev2, theta, kappa, sim, lag, n: int):
        shift = n * theta.detach() * sim.pad_dir
        q, info = sim.step(q_prev.detach(), q_prev2.detach(), shift, float(kappa.detach()), lag)
        ctx.sim, ctx.lag, ctx.n = sim, lag, n
        ctx.save_for_backward(q, theta.detach(), kappa.detach())
        return q

    @staticmethod
    def backward(ctx, qbar):
        q, theta, kappa = ctx.saved_tensors
        sim, lag, n = ctx.sim, ctx.lag, ctx.n
        h2 = sim.h ** 2
        Z = solve_adjoint(sim, q, theta, kappa, lag, n, qbar, ImplicitStep.solver)
        MZ = sim.mass_apply(Z)
        pairs = _system(sim, q, theta, kappa, lag, n)
        _, kin = sim.cs.contact_hvp(q, pairs, Z.contiguous(), lag=lag)
        _, g, _ = sim.cs.eval_contact(q, pairs, lag)
        d_theta = -h2 * n * (kin * sim.pad_dir).sum()
        d_kappa = -h2 * (Z * g).sum() / kappa
        return 2.0 * MZ, -MZ, d_theta, d_kappa, None, None, None


def _segment(q_prev, q_prev2, theta, kappa, sim, lag, n0: int, n1: int):
    for n in range(n0, n1):
        q = ImplicitStep.apply(q_prev, q_prev2, theta, kappa, sim, lag, n)
        q_prev2, q_prev = q_prev, q
    return q_prev, q_prev2


def trajectory_loss(sim, theta, kappa, n_steps: Optional[int] = None, checkpoint_every: Optional[int] = None,
                    solver: str = "dense"):
    """L = ||g_c(q_N)||^2 after N steps with the pad rising by theta per step; theta and
    kappa are 0-d float64 tensors (requires_grad for their derivatives)."""
    N = sim.sc.n_steps if n_steps is None else int(n_steps)
    k = sim.sc.checkpoint_every if checkpoint_every is None else int(checkpoint_every)
    ImplicitStep.solver = solver
    lag = sim.initial_lag(float(kappa.detach()))
    q_prev = sim.q0.clone()
    q_prev2 = sim.q0.clone()
    n0 = 1
    while n0 <= N:
        n1 = N + 1 if k <= 0 else min(N + 1, n0 + k)
        if k > 0 and torch.is_grad_enabled():
            q_prev, q_prev2 = checkpoint(_segment, q_prev, q_prev2, theta, kappa, sim, lag, n0, n1,
                                         use_reentrant=False)
        else:
            q_prev, q_prev2 = _segment(q_prev, q_prev2, theta, kappa, sim, lag, n0, n1)
        n0 = n1
    g = ContactForce.apply(q_prev, theta, kappa, sim, lag, N)
    return (g * g).sum()
