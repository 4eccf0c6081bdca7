"""Literal FP64 restatement of the anisotropic ADE-ELBM on the two-dimensional
nine-velocity tensor-product set D2Q9 (test infrastructure only).

Section 2.1 defines the method on both tensor-product sets, c_i in {-1, 0, 1}^d
with d = 2 or 3, W_i = (2/3)^(d - m_i) (1/6)^(m_i) and c_s^2 = 1/3; Section 4.1 runs
it on D2Q9 with per-node (y-dependent) tensor and velocity fields.  This module
takes the per-node steps of the algorithmic summary (Section 2.7) in the same
order as the three-dimensional oracle in ``oracle.elbm``, with d = 2:
equilibrium (Eq. method-geq), flux/ghost split (Eq. method-lifting), tensorial
flux relaxation with S = (I/2 + D/c_s^2)^-1 (Eq. method-s-from-d), entropic
amplitude (Eqs. method-lambda, method-correction), collision with positivity
fallback (Eqs. method-collision, method-alpha), then streaming (Eq. method-lbe)
with periodic wrap in both axes.

Populations ``g`` have shape ``[9, Ny, Nx]`` (x fastest); vectors ``[2, Ny, Nx]``
or ``[2]``; tensors ``[2, 2]`` or ``[Ny, Nx, 2, 2]``.  Any other trailing node
shape works for the per-node functions.  Readings R1-R6 of ``oracle.elbm``
apply unchanged, with the velocity order i = 3 (cx + 1) + (cy + 1) (rest
population i = 4).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import torch

from .elbm import positivity_fallback

DT = torch.float64
CS2 = 1.0 / 3.0


def _velocity_set():
    """D2Q9: c_i in {-1, 0, 1}^2, W_i = (2/3)^(2 - m_i) (1/6)^(m_i) (Section 2.1)."""
    cs = [(cx, cy) for cx in (-1, 0, 1) for cy in (-1, 0, 1)]
    c = torch.tensor(cs, dtype=DT)
    m = (c != 0).sum(1).to(DT)
    w = (2.0 / 3.0) ** (2.0 - m) * (1.0 / 6.0) ** m
    return c, w, cs


C, W, C_INT = _velocity_set()
Q = 9


def _bcast(vec, like):
    return vec.view((vec.shape[0],) + (1,) * (like.dim() - 1))


def c_dot(v: torch.Tensor) -> torch.Tensor:
    """c_i . v: v [2] -> [9]; v [2, *nodes] -> [9, *nodes]."""
    if v.dim() == 1:
        return C @ v
    return torch.einsum("ia,a...->i...", C, v)


def first_moment(x: torch.Tensor) -> torch.Tensor:
    return torch.einsum("ia,i...->a...", C, x)


def eq_polynomial(u: torch.Tensor) -> torch.Tensor:
    """P_i(u) = 1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u.u/(2 cs2) (Eq. method-geq)."""
    cu = c_dot(u)
    uu = (u * u).sum(0)
    return 1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)


def equilibrium(phi: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """g_i^eq = phi W_i P_i(u)."""
    p = eq_polynomial(u)
    if p.dim() == 1:
        p = _bcast(p, phi.unsqueeze(0))
    return phi.unsqueeze(0) * _bcast(W, phi.unsqueeze(0)) * p


def lift(a: torch.Tensor) -> torch.Tensor:
    """P_i(a) = (W_i / cs2) c_i . a (Eq. method-lifting)."""
    ca = c_dot(a)
    if ca.dim() == 1:
        return W / CS2 * ca
    return _bcast(W, ca) / CS2 * ca


def relaxation_matrix(D: torch.Tensor) -> torch.Tensor:
    """S = (I/2 + D/cs2)^-1 (Eq. method-s-from-d), 2 x 2, exact inverse."""
    return torch.linalg.inv(0.5 * torch.eye(2, dtype=DT) + D / CS2)


def apply_matrix(M: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    if M.dim() == 2:
        return M @ v if v.dim() == 1 else torch.einsum("ab,b...->a...", M, v)
    return torch.einsum("...ab,b...->a...", M, v)


def entropic_amplitude(phi, g_eq, dh, ds_post, u, theta=1e-8, mode="literal"):
    """lambda of Eq. (method-lambda) with C of Eq. (method-correction), guards per R6."""
    valid = (g_eq > 0).all(0) & (phi > 0)
    geq_safe = torch.where(valid.unsqueeze(0), g_eq, torch.ones_like(g_eq))
    hh = (dh * dh / geq_safe).sum(0)
    if mode == "literal":
        hs = (dh * ds_post / geq_safe).sum(0)
        corr = (dh * torch.log(geq_safe / _bcast(W, geq_safe))).sum(0)
    elif mode == "reduced":
        p = eq_polynomial(u)
        if p.dim() == 1:
            p = _bcast(p, dh)
        cu = c_dot(u)
        if cu.dim() == 1:
            cu = _bcast(cu, dh)
        uu = (u * u).sum(0)
        phi_safe = torch.where(valid, phi, torch.ones_like(phi))
        p_safe = torch.where(valid.unsqueeze(0), p.expand_as(dh), torch.ones_like(dh))
        corr = (dh * (torch.log(p_safe) - cu / CS2 + uu / (2.0 * CS2))).sum(0)
        hs = (dh * ds_post * (1.0 / p_safe - 1.0) / _bcast(W, dh)).sum(0) / phi_safe
    else:
        raise ValueError(mode)
    uzero = (u == 0).all(0)
    active = valid & (hh > theta * theta * phi) & ~uzero
    hh_safe = torch.where(active, hh, torch.ones_like(hh))
    return torch.where(active, 1.0 + (hs + corr) / hh_safe, torch.ones_like(hh))


@dataclass
class CollisionInfo:
    lam: torch.Tensor
    alpha: torch.Tensor
    fallback: torch.Tensor


def collide(g, u, S, theta=1e-8, eps=0.0, lam_mode="literal", fallback=True):
    """One collision at every node (Section 2.7, d = 2)."""
    phi = g.sum(0)
    g_eq = equilibrium(phi, u)
    g_neq = g - g_eq
    j = first_moment(g_neq)
    ds = lift(j)
    dh = g_neq - ds
    Sj = apply_matrix(S, j)
    omega_s = -lift(Sj)
    ds_post = ds + omega_s
    lam = entropic_amplitude(phi, g_eq, dh, ds_post, u, theta, lam_mode)
    omega = omega_s - lam.unsqueeze(0) * dh
    if fallback:
        alpha, need = positivity_fallback(g, omega, eps)
    else:
        alpha = torch.ones_like(phi)
        need = torch.zeros_like(phi, dtype=torch.bool)
    return g + alpha.unsqueeze(0) * omega, CollisionInfo(lam=lam, alpha=alpha, fallback=need)


def stream(g_post: torch.Tensor) -> torch.Tensor:
    """g_i(x + c_i, t + 1) = g*_i(x, t), periodic in x and y (Eq. method-lbe)."""
    out = torch.empty_like(g_post)
    for i, (cx, cy) in enumerate(C_INT):
        out[i] = torch.roll(g_post[i], shifts=(cy, cx), dims=(0, 1))
    return out


@dataclass
class Problem:
    u: torch.Tensor                  # [2] or [2, Ny, Nx]
    S: torch.Tensor                  # [2, 2] or [Ny, Nx, 2, 2]
    theta: float = 1e-8
    eps: float = 0.0
    lam_mode: str = "literal"
    fallback: bool = True
    stats: dict = field(default_factory=lambda: dict(fallback_nodes=0, steps=0))

    @staticmethod
    def from_tensor(u, D, **kw) -> "Problem":
        return Problem(u=torch.as_tensor(u, dtype=DT), S=relaxation_matrix(torch.as_tensor(D, dtype=DT)), **kw)


def init_equilibrium(phi0, u) -> torch.Tensor:
    """Reading R2: g = g^eq(phi0, u)."""
    return equilibrium(torch.as_tensor(phi0, dtype=DT), torch.as_tensor(u, dtype=DT))


def step(g: torch.Tensor, prob: Problem) -> torch.Tensor:
    g_post, info = collide(g, prob.u, prob.S, prob.theta, prob.eps, prob.lam_mode, prob.fallback)
    prob.stats["fallback_nodes"] += int(info.fallback.sum())
    prob.stats["steps"] += 1
    return stream(g_post)


def run(g: torch.Tensor, prob: Problem, nsteps: int, callback=None) -> torch.Tensor:
    for n in range(nsteps):
        g = step(g, prob)
        if callback is not None:
            callback(n + 1, g)
    return g


def diagnostics(g: torch.Tensor) -> dict:
    """Mass, entropy H = sum g ln(g/W) over positive g (Eq. method-entropy), min g."""
    pos = g > 0
    gs = torch.where(pos, g, torch.ones_like(g))
    h = torch.where(pos, g * torch.log(gs / _bcast(W, g)), torch.zeros_like(g))
    return dict(mass=float(g.sum()), entropy=float(h.sum()), gmin=float(g.min()))
