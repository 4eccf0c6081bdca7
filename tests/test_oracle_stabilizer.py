"""Pins of the entropic amplitude (Section 2.5, Appendix B) and of the
positivity fallback (Section 2.6).

* lambda is the first-order root of the entropy-stationarity condition
  Eq. (method-entropy-root): solved here exactly (brentq), the gap to the
  oracle's closed form must shrink linearly with the non-equilibrium size.
* u = 0: both numerator terms vanish identically, lambda = 1.
* isotropic limit S = 2 beta I: Omega = -beta (2 ds + gamma dh) with the gamma
  of Appendix B (P8).
* fallback: alpha is the largest step in [0, 1] keeping g + alpha Omega >= eps,
  mass is exact, and an adversarial run stays non-negative (P6)."""
import math

import numpy as np
import pytest
import torch
from scipy.optimize import brentq

import oracle as O

DT = torch.float64
Wn = O.W.numpy()
Cn = O.C.numpy()


def _state(u, delta, seed, n=1):
    """Near-equilibrium nodes: g = g_eq(phi, u) (1 + delta xi) with xi ~ N(0, 1)."""
    g0 = torch.Generator().manual_seed(seed)
    phi = 0.7 + 0.6 * torch.rand(n, generator=g0, dtype=DT)
    geq = O.equilibrium(phi, torch.as_tensor(u, dtype=DT))
    xi = torch.randn(27, n, generator=g0, dtype=DT)
    return geq * (1 + delta * xi)


def _split(g, u, S):
    """Delta h and Delta s_post of one node, from their definitions (numpy)."""
    g = np.asarray(g, float)
    phi = g.sum()
    cu = Cn @ u
    geq = phi * Wn * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u @ u))
    j = Cn.T @ (g - geq)
    dh = g - geq - 3 * Wn * (Cn @ j)
    ds_post = 3 * Wn * (Cn @ ((np.eye(3) - S) @ j))
    return geq, dh, ds_post


def _exact_root(geq, dh, ds_post):
    f = lambda lam: np.sum(dh * np.log((geq + ds_post + (1 - lam) * dh) / Wn))
    # bracket: the arguments must stay positive
    lo, hi = -50.0, 50.0
    ok = lambda lam: np.all(geq + ds_post + (1 - lam) * dh > 0)
    while not ok(lo):
        lo = 0.5 * (lo + 1)
    while not ok(hi):
        hi = 0.5 * (hi + 1)
    return brentq(f, lo, hi, xtol=1e-15, rtol=1e-15)


@pytest.mark.parametrize("mode", ["literal", "reduced"])
def test_lambda_is_first_order_entropy_root(mode):
    u = np.array([0.05, 0.03, 0.02])
    D = np.diag([0.1, 1e-3, 1e-5])
    S = np.linalg.inv(0.5 * np.eye(3) + 3 * D)
    gaps = []
    for delta in (1e-2, 1e-3):
        worst = 0.0
        for seed in range(5):
            g = _state(u, delta, seed)
            _, info = O.collide(g, torch.as_tensor(u), torch.as_tensor(S), theta=0.0, lam_mode=mode,
                                fallback=False)
            lam = info.lam.item()
            geq, dh, dsp = _split(g[:, 0].numpy(), u, S)
            root = _exact_root(geq, dh, dsp)
            worst = max(worst, abs(lam - root) / max(1.0, abs(root)))
        gaps.append(worst)
    # first-order agreement: gap ~ delta
    assert gaps[0] < 5e-2
    assert gaps[1] < 5e-3
    assert gaps[1] < 0.2 * gaps[0]


def test_lambda_literal_equals_reduced():
    u = torch.tensor([0.05, -0.03, 0.02], dtype=DT)
    S = torch.as_tensor(np.linalg.inv(0.5 * np.eye(3) + 3 * np.diag([0.1, 1e-3, 1e-5])))
    g = _state(u.numpy(), 1e-2, 11, n=64)
    _, a = O.collide(g, u, S, theta=0.0, lam_mode="literal")
    _, b = O.collide(g, u, S, theta=0.0, lam_mode="reduced")
    assert torch.allclose(a.lam, b.lam, rtol=1e-10, atol=1e-12)


def test_zero_velocity_gives_lambda_one_identity():
    g = _state(np.zeros(3), 5e-2, 3, n=32)
    u = torch.zeros(3, dtype=DT)
    phi = g.sum(0)
    geq = O.equilibrium(phi, u)
    j = O.first_moment(g - geq)
    dh = g - geq - O.lift(j)
    S = torch.as_tensor(np.linalg.inv(0.5 * np.eye(3) + 3 * np.diag([0.1, 1e-2, 1e-4])))
    dsp = O.lift(O.apply_matrix(torch.eye(3, dtype=DT) - S, j))
    num = (dh * dsp / geq).sum(0) + (dh * torch.log(geq / O.W[:, None])).sum(0)
    assert num.abs().max().item() < 1e-15 * 30
    _, info = O.collide(g, u, S, theta=0.0)
    assert torch.all(info.lam == 1.0)


def test_isotropic_limit_gamma():
    """S = 2 beta I: Omega = -beta (2 ds + gamma dh) with
    gamma = 1/beta - (2 - 1/beta) <dh|ds>_H/<dh|dh>_H + C/(beta <dh|dh>_H)."""
    d = 0.02
    S = np.eye(3) / (0.5 + 3 * d)
    beta = S[0, 0] / 2
    u = np.array([0.04, 0.02, -0.01])
    g = _state(u, 1e-2, 5)
    gpost, info = O.collide(g, torch.as_tensor(u), torch.as_tensor(S), theta=0.0, fallback=False)
    gn = g[:, 0].numpy()
    phi = gn.sum()
    cu = Cn @ u
    geq = phi * Wn * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u @ u))
    j = Cn.T @ (gn - geq)
    ds = 3 * Wn * (Cn @ j)
    dh = gn - geq - ds
    hh = np.sum(dh * dh / geq)
    hs = np.sum(dh * ds / geq)
    corr = np.sum(dh * np.log(geq / Wn))
    gamma = 1 / beta - (2 - 1 / beta) * hs / hh + corr / (beta * hh)
    assert info.lam.item() == pytest.approx(beta * gamma, rel=1e-10)
    omega = gpost[:, 0].numpy() - gn
    assert np.allclose(omega, -beta * (2 * ds + gamma * dh), atol=1e-15)


def test_fallback_alpha_is_maximal_and_mass_exact():
    g0 = torch.Generator().manual_seed(9)
    g = torch.rand(27, 200, generator=g0, dtype=DT) * O.W[:, None]
    g[:, :100] *= torch.rand(27, 100, generator=g0, dtype=DT) ** 4      # rough states
    u = torch.tensor([0.1, 0.0, 0.0], dtype=DT)
    S = torch.as_tensor(np.linalg.inv(0.5 * np.eye(3) + 3 * np.diag([1e-6, 1e-6, 0.2])))
    for eps in (0.0, 1e-6):
        gpost, info = O.collide(g, u, S, theta=1e-8, eps=eps)
        assert info.fallback.any()
        assert torch.allclose(gpost.sum(0), g.sum(0), rtol=1e-14, atol=0)
        # entry states already below eps get alpha = 0 (reading R4) and stay unchanged
        floor = torch.clamp(g.amin(0), max=eps)
        assert (gpost.amin(0) >= floor - 1e-15).all()
        # maximality: a slightly longer step leaves the positive branch
        gfull, _ = O.collide(g, u, S, theta=1e-8, eps=eps, fallback=False)
        omega = gfull - g
        for n in torch.nonzero(info.fallback).flatten()[:40]:
            a = info.alpha[n].item()
            assert 0.0 <= a < 1.0
            longer = g[:, n] + min(1.0, a + 1e-9) * omega[:, n]
            assert (longer < eps).any()
        untouched = ~info.fallback
        assert torch.equal(info.alpha[untouched], torch.ones_like(info.alpha[untouched]))


def test_adversarial_run_stays_nonnegative():
    """Step function, weak diffusivity 1e-6 on two axes, u = 0.1: the fallback
    keeps every population >= 0 and the mass exact."""
    n = 12
    phi0 = np.where(np.arange(n)[None, None, :] < n // 2, 1.0, 1e-3) * np.ones((n, n, n))
    u = torch.tensor([0.1, 0.0, 0.0], dtype=DT)
    D = np.diag([1e-6, 1e-6, 0.2])
    prob = O.Problem.from_tensor(u, D)
    g = O.init_equilibrium(phi0, u)
    m0 = g.sum().item()
    for k in range(20):
        g = O.step(g, prob, k)
        assert g.min().item() >= -1e-17
    assert abs(g.sum().item() - m0) / m0 < 1e-14
    assert prob.stats["fallback_nodes"] > 0


def test_root_mode_solves_stationarity_and_tracks_closed_form():
    """lam_mode='root' zeroes Eq. (method-entropy-root) (checked by evaluating it) and differs
    from the closed form by O(delta)."""
    u = torch.tensor([0.05, 0.03, 0.02], dtype=DT)
    S = torch.as_tensor(np.linalg.inv(0.5 * np.eye(3) + 3 * np.diag([0.1, 1e-3, 1e-5])))
    for delta, bound in ((1e-2, 5e-2), (1e-3, 5e-3)):
        g = _state(u.numpy(), delta, 21, n=16)
        _, a = O.collide(g, u, S, theta=0.0, lam_mode="literal", fallback=False)
        _, b = O.collide(g, u, S, theta=0.0, lam_mode="root", fallback=False)
        assert (a.lam - b.lam).abs().max().item() < bound
        for n in range(16):
            geq, dh, dsp = _split(g[:, n].numpy(), u.numpy(), S.numpy())
            lam = b.lam[n].item()
            res = np.sum(dh * np.log((geq + dsp + (1 - lam) * dh) / Wn))
            assert abs(res) < 1e-14 * np.abs(dh).sum() * 50
