"""Rotated-solid steady conduction (Section 4.2.1, Table 3) on the GPU: Dirichlet x
faces by anti-bounce-back, periodic y and z, uniform rotated conductivity, u = 0.
At steady state the LB flux q = j - S j / 2 over the gradient G_x recovers the
conductivity column K_{.x}; the entries are compared with Table 3's exact values.

Lattice diffusivity = 1e-3 x conductivity; 128 nodes in x (as the paper); the
solution is y/z-uniform, so 4 x 4 nodes across suffice.  Shifted temperatures
(2, 1) keep every population positive."""
import json
import os

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import gpu_lattice

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))["table3_rotated_solid"]


@pytest.fixture(scope="module")
def E():
    from paper_2605_01774_gb300 import elbm
    elbm.lib()
    return elbm


@pytest.mark.parametrize("row", GOLD["rows"])
def test_table3_conductivities_from_lb_flux(E, row):
    scale = 1e-3
    K = synth.tensor_from_principal(row["k"], synth.rot_zyz_deg(*row["euler_deg"]))
    dims = (128, 4, 4)
    lat = gpu_lattice(E, dims, "f64", D=K * scale, bc=(2.0, 1.0))
    x = np.arange(128)
    phi0 = np.broadcast_to(2.0 - (x + 0.5) / 128, dims[::-1]).copy()
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    phi = torch.empty(dims[::-1], dtype=torch.float64, device="cuda")
    q = torch.empty((3,) + dims[::-1], dtype=torch.float64, device="cuda")
    prev = None
    for chunk in range(60):
        E.elbm_step(lat.h, 20000)
        E.elbm_read_moments(lat.h, phi, q)
        torch.cuda.synchronize()
        cur = q.clone()
        if prev is not None and (cur - prev).abs().max().item() < 1e-15:
            break
        prev = cur
    d = E.elbm_reduce(lat.h)
    lat.close()
    G = 1.0 / 128
    K_rec = q[:, 0, 0, 8:120].mean(-1).cpu().numpy() / G / scale
    lin = np.abs(phi.cpu().numpy()[0, 0] - (2.0 - (x + 0.5) / 128)).max()
    print(f"k={row['k']} angles={row['euler_deg']}: K_rec {K_rec} exact {K[:, 0]} linear-profile err {lin:.1e} "
          f"steps {(chunk + 1) * 20000}")
    assert d["n_fallback"] == 0
    assert lin < 1e-10
    assert np.allclose(K_rec, K[:, 0], rtol=1e-8, atol=1e-9)
    assert np.allclose(K_rec, row["K_exact"], atol=6e-4)
