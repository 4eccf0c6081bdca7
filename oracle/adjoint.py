"""FP64 CPU reference for gradients of a concentration misfit with respect to
per-node tensor parameters (test infrastructure only).

theta [6, Nz, Ny, Nx] = (ln d1, ln d2, ln d3, ZYZ angles a, b, c) ->
D = R diag(exp(l)) R^T -> S (Eq. method-s-from-d) -> the oracle's step
(Section 2.7) from g_eq(phi0, u).  J = 1/2 sum_{t in obs} sum_x (phi_t - phi*_t)^2.
The gradient is torch's reverse-mode differentiation of this literal program
(no hand-written derivative), optionally with torch.utils.checkpoint segments.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint

from . import elbm as O


def _segment(g, prob, t0, t1):
    for n in range(t0, t1):
        g = O.step(g, prob, n)
    return g


def misfit(theta, phi0, u, nsteps, obs, targets, guard=1e-8, lam_mode="literal", segment=None):
    """J(theta) as a differentiable torch scalar; targets is a dict t -> phi*_t."""
    u = torch.as_tensor(u, dtype=O.DT)
    S = O.relaxation_matrix(O.tensor_from_params(theta))
    prob = O.Problem(u=u, S=S, theta=guard, lam_mode=lam_mode)
    g = O.init_equilibrium(phi0, u)
    J = torch.zeros((), dtype=O.DT)
    t = 0
    stops = sorted(set(obs) | set(range(segment, nsteps, segment) if segment else []) | {nsteps})
    for stop in stops:
        if segment:
            g = checkpoint(_segment, g, prob, t, stop, use_reentrant=False)
        else:
            g = _segment(g, prob, t, stop)
        t = stop
        if t in obs:
            J = J + 0.5 * ((g.sum(0) - torch.as_tensor(targets[t], dtype=O.DT)) ** 2).sum()
    return J, prob


def misfit_gradient(theta, phi0, u, nsteps, obs, targets, guard=1e-8, segment=None):
    th = torch.as_tensor(theta, dtype=O.DT).clone().requires_grad_(True)
    J, prob = misfit(th, phi0, u, nsteps, obs, targets, guard=guard, segment=segment)
    J.backward()
    return float(J.detach()), th.grad.detach(), prob.stats["fallback_nodes"]


def forward_snapshots(theta, phi0, u, nsteps, obs, guard=1e-8):
    """phi at the observation steps (used to build synthetic targets)."""
    u = torch.as_tensor(u, dtype=O.DT)
    S = O.relaxation_matrix(O.tensor_from_params(torch.as_tensor(theta, dtype=O.DT)))
    prob = O.Problem(u=u, S=S, theta=guard)
    g = O.init_equilibrium(phi0, u)
    out = {}
    for n in range(nsteps):
        g = O.step(g, prob, n)
        if n + 1 in obs:
            out[n + 1] = g.sum(0).clone()
    return out
