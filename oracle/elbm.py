"""Literal FP64 restatement of the anisotropic ADE-ELBM (test infrastructure only).

Arrays are torch float64 CPU tensors.  Populations ``g`` have shape
``[27, Nz, Ny, Nx]`` (x fastest).  Vectors on the lattice (u, j, a) have shape
``[3, Nz, Ny, Nx]`` or ``[3]`` when uniform.  Tensors (D, S) have shape
``[3, 3]`` (uniform) or ``[Nz, Ny, Nx, 3, 3]`` (per node).  Every function
also accepts any other trailing node shape (e.g. ``[27, M]`` for M sampled
nodes), which the tests use to evaluate single nodes.

The per-node order of operations follows the algorithmic summary of
Section 2.7: equilibrium, tensor map and flux/ghost split, tensorial flux
relaxation, entropic amplitude, collision with positivity fallback, stream.

Readings (where the paper is silent or ambiguous):

R1  Velocity order: i = 9 (cx+1) + 3 (cy+1) + (cz+1); rest population i = 13.
R2  Initial populations: the equilibrium g_i = g_i^eq(phi0, u), i.e. j = 0.
R3  Eq. (method-update) is read as "collide at the node, then stream" (Eq. method-lbe).
R4  Fallback: alpha is evaluated only when some g_i + Omega_i < eps, as
    alpha = clamp(min_{Omega_i<0} (g_i - eps)/(-Omega_i), 0, 1).
R5  eps is an absolute threshold, default 0.
R6  Entropic amplitude: lambda = 1 where u = 0 exactly (there both numerator
    terms of Eq. method-lambda vanish identically: sum_i dh_i = 0 and
    sum_i c_i dh_i = 0), and lambda = 1 where <dh|dh>_H <= theta^2 phi (the
    "dh = 0" rule of Eq. method-lambda given a threshold), or where phi or a
    g_i^eq is not positive (the H-product and the logarithm are undefined).
    Mode "literal" evaluates Eqs. (method-lambda, method-correction) as
    printed; mode "reduced" drops the terms that are identically zero:
    C = sum_i dh_i (ln P_i(u) - c_i.u/cs2 + u.u/(2 cs2)) and
    <dh|ds_post>_H = sum_i dh_i ds_post_i (1/P_i - 1) / (W_i phi).
R7  Dirichlet faces (Section 4.2.1 gives no scheme): halfway anti-bounce-back
    at x = -1/2 and x = Nx - 1/2:
    g_i(x_b, t+1) = -g*_opp(i)(x_b, t) + 2 W_i phi_w (1 + (c_i.u_w)^2/(2 cs2^2) - u_w.u_w/(2 cs2)).
R8  Source (Section 3.3): Strang split S(1/2) -> T -> S(1/2), half-step
    g_i += (1/2) R E_i(u) with E_i(u) = W_i P_i(u); the stored state after a
    step is the one after the trailing half-step.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import torch

DT = torch.float64
CS2 = 1.0 / 3.0          # c_s^2 = c^2/3 with c = dx/dt = 1 (Section 2.1)


def _velocity_set():
    """D3Q27 tensor-product velocity set and weights (Section 2.1).

    c_i in {-1, 0, 1}^3, W_i = (2/3)^(3-m_i) (1/6)^(m_i), m_i = number of
    non-zero components.
    """
    cs = [(cx, cy, cz) for cx in (-1, 0, 1) for cy in (-1, 0, 1) for cz in (-1, 0, 1)]
    c = torch.tensor(cs, dtype=DT)
    m = (c != 0).sum(1).to(DT)
    w = (2.0 / 3.0) ** (3.0 - m) * (1.0 / 6.0) ** m
    opp = torch.tensor([cs.index((-a, -b, -d)) for (a, b, d) in cs], dtype=torch.long)
    return c, w, opp, cs


C, W, OPP, C_INT = _velocity_set()
Q = 27


def _bcast(vec: torch.Tensor, like: torch.Tensor) -> torch.Tensor:
    """View a [27] vector so it broadcasts against [27, *nodes]."""
    return vec.view((vec.shape[0],) + (1,) * (like.dim() - 1))


# ----------------------------------------------------------------------------
# Moments, equilibrium, lift (Sections 2.1 and 2.2)
# ----------------------------------------------------------------------------
def c_dot(v: torch.Tensor) -> torch.Tensor:
    """c_i . v for all i: v [3] -> [27]; v [3, *nodes] -> [27, *nodes]."""
    if v.dim() == 1:
        return C @ v
    return torch.einsum("ia,a...->i...", C, v)


def zeroth_moment(g: torch.Tensor) -> torch.Tensor:
    """phi = sum_i g_i."""
    return g.sum(0)


def first_moment(x: torch.Tensor) -> torch.Tensor:
    """sum_i c_i x_i -> [3, *nodes]."""
    return torch.einsum("ia,i...->a...", C, x)


def eq_polynomial(u: torch.Tensor) -> torch.Tensor:
    """P_i(u) = 1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u.u/(2 cs2) (Eq. method-geq)."""
    cu = c_dot(u)
    uu = (u * u).sum(0)
    return 1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)


def equilibrium(phi: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """g_i^eq = phi W_i P_i(u) (Eq. method-geq)."""
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


# ----------------------------------------------------------------------------
# Tensor map (Section 2.3)
# ----------------------------------------------------------------------------
def relaxation_matrix(D: torch.Tensor) -> torch.Tensor:
    """S = (I/2 + D/(cs2 dt))^{-1} with dt = 1 (Eq. method-s-from-d); exact 3x3 inverse."""
    eye = torch.eye(3, dtype=DT)
    return torch.linalg.inv(0.5 * eye + D / CS2)


def diffusion_from_relaxation(S: torch.Tensor) -> torch.Tensor:
    """D = cs2 dt (S^{-1} - I/2) (Eq. method-d-from-s)."""
    eye = torch.eye(3, dtype=DT)
    return CS2 * (torch.linalg.inv(S) - 0.5 * eye)


def apply_matrix(M: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    """(M v) per node: M [3,3] or [*nodes,3,3]; v [3, *nodes] -> [3, *nodes]."""
    if M.dim() == 2:
        if v.dim() == 1:
            return M @ v
        return torch.einsum("ab,b...->a...", M, v)
    return torch.einsum("...ab,b...->a...", M, v)


# ----------------------------------------------------------------------------
# Entropic amplitude (Section 2.5) and positivity fallback (Section 2.6)
# ----------------------------------------------------------------------------
def entropic_amplitude(phi, g_eq, dh, ds_post, u, theta=1e-8, mode="literal"):
    """lambda of Eq. (method-lambda) with the correction C of Eq. (method-correction).

    <x|y>_H = sum_i x_i y_i / g_i^eq.  Guards per reading R6.  Returns lambda
    with the node shape of phi.
    """
    valid = (g_eq > 0).all(0) & (phi > 0)
    geq_safe = torch.where(valid.unsqueeze(0), g_eq, torch.ones_like(g_eq))
    hh = (dh * dh / geq_safe).sum(0)                       # <dh|dh>_H
    if mode == "literal":
        hs = (dh * ds_post / geq_safe).sum(0)              # <dh|ds_post>_H
        corr = (dh * torch.log(geq_safe / _bcast(W, geq_safe))).sum(0)   # C
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
    lam = torch.where(active, 1.0 + (hs + corr) / hh_safe, torch.ones_like(hh))
    return lam


def entropy_root(g_eq, dh, ds_post, lam0):
    """Exact root of Eq. (method-entropy-root) at each node where lam0 is not exactly 1:
    sum_i dh_i ln((g_eq_i + ds_post_i + (1 - lam) dh_i) / W_i) = 0, by scipy's brentq on
    the open bracket where every argument is positive (the function decreases from +inf to
    -inf across it).  Nodes whose bracket is empty keep lam0.  (parity: the GPU's FP64
    Newton solves the same equation.)"""
    import numpy as np
    from scipy.optimize import brentq
    ge = g_eq.reshape(27, -1).double().numpy()
    dh_ = dh.reshape(27, -1).double().numpy()
    dp = ds_post.reshape(27, -1).double().numpy()
    l0 = lam0.reshape(-1).double().numpy().copy()
    w = W.numpy()
    out = l0.copy()
    for n in range(l0.size):
        if l0[n] == 1.0:
            continue
        b = ge[:, n] + dp[:, n]
        d = dh_[:, n]
        pos, neg = d > 0, d < 0
        if np.any(~pos & ~neg & ~(b > 0)) or not pos.any() or not neg.any():
            continue
        hi = np.min(1.0 + b[pos] / d[pos])
        lo = np.max(1.0 + b[neg] / d[neg])
        if not lo < hi:
            continue
        f = lambda lam: float(np.sum(d * np.log((b + (1.0 - lam) * d) / w)))
        span = hi - lo
        a_, b_ = lo + 1e-13 * span, hi - 1e-13 * span
        if not (f(a_) > 0 > f(b_)):
            continue
        out[n] = brentq(f, a_, b_, xtol=1e-15, rtol=1e-15, maxiter=500)
    return torch.as_tensor(out, dtype=DT).reshape(lam0.shape)


def positivity_fallback(g: torch.Tensor, omega: torch.Tensor, eps: float = 0.0):
    """alpha of Eq. (method-alpha) under reading R4.  Returns (alpha, triggered)."""
    need = ((g + omega) < eps).any(0)
    neg = omega < 0
    denom = torch.where(neg, -omega, torch.ones_like(omega))
    ratio = torch.where(neg, (g - eps) / denom, torch.full_like(omega, math.inf))
    a = ratio.amin(0).clamp(0.0, 1.0)
    alpha = torch.where(need, a, torch.ones_like(a))
    return alpha, need


@dataclass
class CollisionInfo:
    lam: torch.Tensor
    alpha: torch.Tensor
    fallback: torch.Tensor


def collide(g: torch.Tensor, u: torch.Tensor, S: torch.Tensor, theta: float = 1e-8,
            eps: float = 0.0, lam_mode: str = "literal", fallback: bool = True):
    """One collision at every node, steps 1-5 of the algorithmic summary.

    Returns (g_post, CollisionInfo).  u is [3] or [3, *nodes]; S is [3,3] or
    [*nodes, 3, 3].
    """
    phi = zeroth_moment(g)
    g_eq = equilibrium(phi, u)                       # step 1, Eq. method-geq
    g_neq = g - g_eq                                 # step 2
    j = first_moment(g_neq)                          # Eq. method-first-moment
    ds = lift(j)                                     # Eq. method-lifting
    dh = g_neq - ds
    Sj = apply_matrix(S, j)                          # step 3, Eq. method-flux-relaxation
    omega_s = -lift(Sj)
    ds_post = ds + omega_s                           # = P((I - S) j)
    lam = entropic_amplitude(phi, g_eq, dh, ds_post, u, theta,
                             "literal" if lam_mode == "root" else lam_mode)          # step 4
    if lam_mode == "root":
        lam = entropy_root(g_eq, dh, ds_post, lam)       # Eq. method-entropy-root, exactly
    omega = omega_s - lam.unsqueeze(0) * dh          # step 5, Eq. method-collision
    if fallback:
        alpha, need = positivity_fallback(g, omega, eps)   # Eq. method-alpha
    else:
        alpha = torch.ones_like(phi)
        need = torch.zeros_like(phi, dtype=torch.bool)
    g_post = g + alpha.unsqueeze(0) * omega          # Eq. method-update
    return g_post, CollisionInfo(lam=lam, alpha=alpha, fallback=need)


# ----------------------------------------------------------------------------
# Streaming (Eq. method-lbe), boundaries and source
# ----------------------------------------------------------------------------
def stream(g_post: torch.Tensor, dirichlet_x=None, u_wall=None) -> torch.Tensor:
    """g_i(x + c_i, t + 1) = g*_i(x, t); periodic in every axis, or with
    anti-bounce-back x-faces (reading R7) when dirichlet_x = (phi_lo, phi_hi)."""
    out = torch.empty_like(g_post)
    nx = g_post.shape[-1]
    if dirichlet_x is not None:
        uw = torch.zeros(3, dtype=DT) if u_wall is None else torch.as_tensor(u_wall, dtype=DT)
        cuw = C @ uw
        even = 1.0 + cuw * cuw / (2.0 * CS2 * CS2) - (uw * uw).sum() / (2.0 * CS2)
    for i, (cx, cy, cz) in enumerate(C_INT):
        r = torch.roll(g_post[i], shifts=(cz, cy), dims=(0, 1))
        if dirichlet_x is None:
            out[i] = torch.roll(r, shifts=cx, dims=2)
            continue
        o = OPP[i]
        if cx == 0:
            out[i] = r
        elif cx == 1:
            out[i, :, :, 1:] = r[:, :, :-1]
            out[i, :, :, 0] = -g_post[o, :, :, 0] + 2.0 * W[i] * dirichlet_x[0] * even[i]
        else:
            out[i, :, :, :-1] = r[:, :, 1:]
            out[i, :, :, nx - 1] = -g_post[o, :, :, nx - 1] + 2.0 * W[i] * dirichlet_x[1] * even[i]
    return out


def source_half_step(g: torch.Tensor, R: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """g_i += (dt/2) R E_i(u), E_i(u) = W_i P_i(u) (Section 3.3)."""
    E = W * eq_polynomial(u) if u.dim() == 1 else _bcast(W, g) * eq_polynomial(u)
    if E.dim() == 1:
        E = _bcast(E, g)
    return g + 0.5 * R.unsqueeze(0) * E


# ----------------------------------------------------------------------------
# Problems and runs
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    """One lattice problem: velocity, tensor, boundaries, source and guards."""
    u: torch.Tensor                       # [3] or [3, Nz, Ny, Nx]
    S: torch.Tensor                       # [3, 3] or [Nz, Ny, Nx, 3, 3]
    dirichlet_x: Optional[tuple] = None
    source: Optional[object] = None       # tensor [Nz, Ny, Nx] or callable(t_mid) -> tensor
    theta: float = 1e-8
    eps: float = 0.0
    lam_mode: str = "literal"
    fallback: bool = True
    stats: dict = field(default_factory=lambda: dict(fallback_nodes=0, steps=0))

    @staticmethod
    def from_tensor(u, D, **kw) -> "Problem":
        u = torch.as_tensor(u, dtype=DT)
        D = torch.as_tensor(D, dtype=DT)
        return Problem(u=u, S=relaxation_matrix(D), **kw)


def init_equilibrium(phi0, u) -> torch.Tensor:
    """Reading R2: g = g^eq(phi0, u)."""
    return equilibrium(torch.as_tensor(phi0, dtype=DT), torch.as_tensor(u, dtype=DT))


def _source_at(prob: Problem, t_mid: float):
    if prob.source is None:
        return None
    if callable(prob.source):
        return prob.source(t_mid)
    return prob.source


def step(g: torch.Tensor, prob: Problem, n: int = 0) -> torch.Tensor:
    """One collide-stream step from time n to n + 1 (with the Strang source if any)."""
    R = _source_at(prob, n + 0.5)
    if R is not None:
        g = source_half_step(g, R, prob.u)
    g_post, info = collide(g, prob.u, prob.S, prob.theta, prob.eps, prob.lam_mode, prob.fallback)
    prob.stats["fallback_nodes"] += int(info.fallback.sum())
    prob.stats["steps"] += 1
    g = stream(g_post, prob.dirichlet_x)
    if R is not None:
        g = source_half_step(g, R, prob.u)
    return g


def run(g: torch.Tensor, prob: Problem, nsteps: int, t0: int = 0, callback=None) -> torch.Tensor:
    for n in range(t0, t0 + nsteps):
        g = step(g, prob, n)
        if callback is not None:
            callback(n + 1, g)
    return g


def flux_q(g: torch.Tensor, u: torch.Tensor, S: torch.Tensor) -> torch.Tensor:
    """LB diffusive flux q = j - (1/2) S j from the pre-collision state (Eq. app-cube-lb-flux)."""
    phi = zeroth_moment(g)
    j = first_moment(g - equilibrium(phi, u))
    return j - 0.5 * apply_matrix(S, j)


def diagnostics(g: torch.Tensor) -> dict:
    """Mass sum(phi), entropy H = sum g ln(g/W) (Eq. method-entropy) over positive g, min g."""
    pos = g > 0
    gs = torch.where(pos, g, torch.ones_like(g))
    h = torch.where(pos, g * torch.log(gs / _bcast(W, g)), torch.zeros_like(g))
    return dict(mass=float(g.sum()), entropy=float(h.sum()), gmin=float(g.min()))


# ----------------------------------------------------------------------------
# Per-node tensor parametrisation (3 log-eigenvalues + ZYZ angles)
# ----------------------------------------------------------------------------
def rotation_zyz(a: torch.Tensor, b: torch.Tensor, c: torch.Tensor) -> torch.Tensor:
    """R = Rz(a) Ry(b) Rz(c) per node -> [*nodes, 3, 3] (Section 3.1 convention)."""
    one, zero = torch.ones_like(a), torch.zeros_like(a)

    def rz(t):
        ct, st = torch.cos(t), torch.sin(t)
        return torch.stack([torch.stack([ct, -st, zero], -1),
                            torch.stack([st, ct, zero], -1),
                            torch.stack([zero, zero, one], -1)], -2)

    def ry(t):
        ct, st = torch.cos(t), torch.sin(t)
        return torch.stack([torch.stack([ct, zero, st], -1),
                            torch.stack([zero, one, zero], -1),
                            torch.stack([-st, zero, ct], -1)], -2)

    return rz(a) @ ry(b) @ rz(c)


def tensor_from_params(theta: torch.Tensor) -> torch.Tensor:
    """D = R diag(exp(l1), exp(l2), exp(l3)) R^T from theta [6, *nodes] -> [*nodes, 3, 3]."""
    R = rotation_zyz(theta[3], theta[4], theta[5])
    d = torch.exp(theta[0:3]).movedim(0, -1)
    return R @ torch.diag_embed(d) @ R.transpose(-1, -2)
