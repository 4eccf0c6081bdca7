"""Pins of the D2Q9 oracle (oracle.d2q9) against what the paper and the mathematics fix:
the weights printed in Section 2.1, the quadrature and lift identities, the exact Fourier
recurrence of the zero-velocity scheme (derived independently in fourier_pin), the continuum
decay law exp(-k.Dk t), the analytic anisotropic Gaussian (centroid u t, covariance growth
2 D t), exact mass under the positivity fallback, and the isotropic limit."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle.d2q9 as O2
import synth
from fourier_pin import dominant_rate_2d, mode_history_2d

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def _rot2(a):
    return np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])


def _tensor2(d, a):
    R = _rot2(a)
    return R @ np.diag(d) @ R.T


def _grid2(nx, ny):
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    return x, y


def test_weights_are_the_printed_ones():
    """Section 2.1: D2Q9 weights 4/9 (rest), 1/9 (axis), 1/36 (diagonal)."""
    printed = [float(Fraction(v)) for v in GOLD["d3q27_weights"]["d2q9_by_m"]]
    m = (O2.C != 0).sum(1)
    for i in range(9):
        assert O2.W[i].item() == pytest.approx(printed[int(m[i])], rel=1e-15)
    assert O2.C_INT[4] == (0, 0)


def test_quadrature_and_equilibrium_moments():
    c, w = O2.C.numpy(), O2.W.numpy()
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(c.T @ w, 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(2) / 3, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    # fourth moment of the tensor product: 1/3 on x^4, 1/9 on x^2 y^2 (isotropic 1/9 (dd + dd + dd))
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    assert m4[0, 0, 0, 0] == pytest.approx(1 / 3) and m4[0, 0, 1, 1] == pytest.approx(1 / 9)
    u = torch.tensor([0.05, -0.03], dtype=torch.float64)
    geq = O2.equilibrium(torch.tensor(0.8, dtype=torch.float64), u).numpy()
    assert geq.sum() == pytest.approx(0.8, rel=1e-15)
    assert np.allclose(c.T @ geq, 0.8 * u.numpy(), atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", geq, c, c), 0.8 * (np.eye(2) / 3 + np.outer(u, u)), atol=1e-16)


def test_lift_and_split_identities():
    a = torch.tensor([0.3, -0.7], dtype=torch.float64)
    p = O2.lift(a)
    assert abs(p.sum().item()) < 1e-16
    assert np.allclose(O2.first_moment(p).numpy(), a.numpy(), atol=1e-16)
    rng = np.random.default_rng(0)
    g = torch.as_tensor(rng.uniform(0.1, 1.0, (9, 3, 4)))
    u = torch.tensor([0.04, 0.02], dtype=torch.float64)
    phi = g.sum(0)
    gneq = g - O2.equilibrium(phi, u)
    j = O2.first_moment(gneq)
    dh = gneq - O2.lift(j)
    assert (dh.sum(0).abs() / phi).max().item() < 1e-15          # rounding of phi-sized sums
    assert (O2.first_moment(dh).abs() / phi).max().item() < 1e-15


@pytest.mark.parametrize("dims,m,d,a", [((12, 10), (1, 2), (0.05, 0.005), 0.7), ((9, 7), (2, -1), (0.1, 1e-4), 2.1),
                                        ((32, 32), (1, 1), (0.05, 0.0005), 0.3)])
def test_exact_fourier_recurrence_2d(dims, m, d, a):
    """Non-square grids and oblique modes: swapped axes or streaming signs break it."""
    nx, ny = dims
    x, y = _grid2(nx, ny)
    k = 2 * math.pi * np.array([m[0] / nx, m[1] / ny])
    phi0 = 1.0 + 0.1 * np.sin(k[0] * x + k[1] * y)
    D = _tensor2(d, a)
    prob = O2.Problem.from_tensor((0.0, 0.0), D)
    g = O2.init_equilibrium(phi0, (0.0, 0.0))
    idx = (m[1] % ny, m[0] % nx)
    hist = []
    O2.run(g, prob, 60, callback=lambda n, g: hist.append(np.fft.fft2(g.sum(0).numpy())[idx]))
    S = np.linalg.inv(0.5 * np.eye(2) + 3.0 * D)
    pred = mode_history_2d(k, S, np.fft.fft2(phi0)[idx], 60)
    assert np.max(np.abs(np.array(hist) - pred)) / abs(np.fft.fft2(phi0)[idx]) < 1e-12
    assert prob.stats["fallback_nodes"] == 0


def test_continuum_decay_rate_2d():
    """32^2, k = 2 pi (1, 1)/32: the exact rate of the scheme is within 1e-2 of k.Dk."""
    D = _tensor2((0.05, 0.005), 0.4)
    k = 2 * math.pi * np.array([1, 1]) / 32
    S = np.linalg.inv(0.5 * np.eye(2) + 3.0 * D)
    theory = k @ D @ k
    assert abs(dominant_rate_2d(k, S) - theory) / theory < 1e-2


def test_gaussian_plume_2d():
    """Analytic anisotropic Gaussian: centroid speed u, covariance growth 2 D t, exact mass."""
    nx = ny = 48
    x, y = _grid2(nx, ny)
    mu0 = np.array([23.5, 23.5])
    phi0 = np.exp(-((x - mu0[0]) ** 2 + (y - mu0[1]) ** 2) / (2 * 5.0 ** 2))
    u = np.array([0.05, -0.03])
    D = _tensor2((0.05, 0.005), 0.6)
    prob = O2.Problem.from_tensor(u, D)
    snaps = {}
    O2.run(O2.init_equilibrium(phi0, u), prob, 80,
           callback=lambda n, g: snaps.__setitem__(n, g.sum(0).numpy()) if n in (40, 80) else None)

    def moments(phi, center):
        X = [x, y]
        N = [nx, ny]
        dd = [((X[a] - center[a] + N[a] / 2) % N[a]) - N[a] / 2 for a in range(2)]
        M = phi.sum()
        mu = np.array([(phi * dd[a]).sum() / M for a in range(2)])
        cov = np.array([[(phi * (dd[a] - mu[a]) * (dd[b] - mu[b])).sum() / M for b in range(2)] for a in range(2)])
        return M, mu + center, cov

    m1 = moments(snaps[40], mu0 + 40 * u)
    m2 = moments(snaps[80], mu0 + 80 * u)
    assert abs(m2[0] - phi0.sum()) / phi0.sum() < 1e-13
    assert np.abs((m2[1] - m1[1]) / 40 - u).max() < 1e-4
    D_rec = (m2[2] - m1[2]) / 80.0
    assert np.abs(D_rec - D).max() / np.abs(D).max() < 1e-2


def test_fallback_keeps_mass_and_positivity_2d():
    """Adversarial step function with a weak axis (Eq. method-alpha): populations stay >= 0
    and the mass is exact to rounding."""
    nx, ny = 16, 12
    x, y = _grid2(nx, ny)
    phi0 = np.where(x < 8, 1.0, 1e-6)
    prob = O2.Problem.from_tensor((0.1, 0.05), _tensor2((0.05, 1e-6), 0.5), theta=1e-8)
    g = O2.init_equilibrium(phi0, (0.1, 0.05))
    M0 = float(g.sum())
    for _ in range(30):
        g = O2.step(g, prob)
        assert float(g.min()) >= 0.0
    assert abs(float(g.sum()) - M0) / M0 < 1e-13
    assert prob.stats["fallback_nodes"] > 0


def test_isotropic_limit_2d():
    """S = 2 beta I (isotropic D): the collision is Omega = -beta (2 ds + gamma dh) with
    gamma = lambda / beta, i.e. the flux part relaxes at rate 2 beta (Appendix B)."""
    beta = 0.8
    D = (1.0 / (2 * beta) - 0.5) / 3.0 * np.eye(2)
    S = O2.relaxation_matrix(torch.as_tensor(D)).numpy()
    assert np.allclose(S, 2 * beta * np.eye(2), atol=1e-15)
    rng = np.random.default_rng(5)
    g = torch.as_tensor(rng.uniform(0.05, 0.2, (9, 4)))
    u = torch.tensor([0.02, 0.01], dtype=torch.float64)
    gp, info = O2.collide(g, u, torch.as_tensor(S), theta=0.0, fallback=False)
    phi = g.sum(0)
    gneq = g - O2.equilibrium(phi, u)
    ds = O2.lift(O2.first_moment(gneq))
    dh = gneq - ds
    assert np.allclose((gp - g).numpy(), (-2 * beta * ds - info.lam * dh).numpy(), atol=1e-16)
