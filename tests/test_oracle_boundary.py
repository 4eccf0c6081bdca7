"""Pins of the Dirichlet faces (reading R7, anti-bounce-back) and of the
Strang-split source (Section 3.3).

P7: for u = 0, a uniform rotated tensor, Dirichlet x-faces and periodic y/z,
the steady state is the linear profile and the LB flux q = j - S j / 2 equals
K_{.x} G_x (Section 4.2.1); the recovered entries reproduce Table 3's exact
conductivities.  The oracle's steady state is computed exactly as the fixed
point of its own affine step map (u = 0 makes lambda = 1, so the map is affine
without the fallback)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
DT = torch.float64


def _fixed_point(prob, dims):
    nx, ny, nz = dims
    n = 27 * nx * ny * nz
    b = O.step(torch.zeros(27, nz, ny, nx, dtype=DT), prob).flatten()
    T = torch.empty(n, n, dtype=DT)
    for k in range(n):
        e = torch.zeros(n, dtype=DT)
        e[k] = 1.0
        T[:, k] = O.step(e.view(27, nz, ny, nx), prob).flatten() - b
    return torch.linalg.solve(torch.eye(n, dtype=DT) - T, b).view(27, nz, ny, nx)


@pytest.mark.parametrize("row", GOLD["table3_rotated_solid"]["rows"])
def test_steady_conduction_table3(row):
    scale = 1e-3                       # lattice diffusivity = 1e-3 x conductivity
    K = synth.tensor_from_principal(row["k"], synth.rot_zyz_deg(*row["euler_deg"]))
    nx = 8
    # shifted scalar (Section 3.3): T_h = 2, T_c = 1 keeps every population positive
    prob = O.Problem.from_tensor(np.zeros(3), K * scale, dirichlet_x=(2.0, 1.0), fallback=False)
    g = _fixed_point(prob, (nx, 1, 1))
    assert g.min().item() > 0
    phi = g.sum(0)[0, 0].numpy()
    x = np.arange(nx)
    assert np.abs(phi - (2.0 - (x + 0.5) / nx)).max() < 1e-13       # linear profile, walls at -1/2, Nx-1/2
    q = O.flux_q(g, torch.zeros(3, dtype=DT), prob.S)[:, 0, 0, :].numpy()
    G = 1.0 / nx
    K_rec = q / G / scale
    assert np.abs(K_rec - K[:, :1]).max() / np.abs(K).max() < 1e-12
    assert np.allclose(K_rec[:, 3], row["K_exact"], atol=6e-4)
    # the same state is a fixed point of the full step with the fallback enabled
    prob_fb = O.Problem.from_tensor(np.zeros(3), K * scale, dirichlet_x=(2.0, 1.0))
    assert (O.step(g, prob_fb) - g).abs().max().item() < 1e-15


def test_steady_conduction_3d_grid_is_y_z_uniform():
    """Same fixed point on a 6 x 3 x 2 grid: y/z-periodic axes carry no structure."""
    K = synth.tensor_from_principal((100, 10, 0.01), synth.rot_zyz_deg(135, 35, 75)) * 1e-3
    prob = O.Problem.from_tensor(np.zeros(3), K, dirichlet_x=(0.3, 1.2), fallback=False)
    g = _fixed_point(prob, (6, 3, 2))
    phi = g.sum(0).numpy()
    x = np.arange(6)
    assert np.abs(phi - (0.3 + 0.9 * (x + 0.5) / 6)[None, None, :]).max() < 1e-13


def test_source_mass_balance_and_split():
    """Periodic box, u != 0, time-constant R: mass grows by sum(R) per step, and
    the half-steps use E_i(u) = W_i P_i(u) (sum_i E_i = 1, sum_i c_i E_i = u)."""
    wl = synth.gaussian_plume(n=12, sigma0=3.0, eig=(0.02, 0.005, 0.001), steps=5)
    R = 1e-3 * synth.gaussian(wl.dims, (5.5, 5.5, 5.5), 2.0)
    prob = O.Problem.from_tensor(wl.u, wl.D, source=torch.as_tensor(R))
    g = O.init_equilibrium(0.1 + wl.phi0, wl.u)
    m0 = g.sum().item()
    g = O.run(g, prob, 5)
    assert g.sum().item() - m0 == pytest.approx(5 * R.sum(), rel=1e-11)
    gh = O.source_half_step(torch.zeros(27, 1, dtype=DT), torch.ones(1, dtype=DT), torch.as_tensor(wl.u))
    assert gh.sum().item() == pytest.approx(0.5, abs=1e-15)
    assert np.allclose(O.first_moment(gh)[:, 0].numpy(), 0.5 * wl.u, atol=1e-16)
