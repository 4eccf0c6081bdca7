"""Pins of the oracle's tensor parametrisation and conservation diagnostics.

* ``tensor_from_params`` (with ``rotation_zyz``): theta = (ln d1, ln d2, ln d3, a, b, c) must
  give D = R diag(d) R^T with the paper's ZYZ convention.  The paper prints the resulting
  Cartesian tensors: Table 1 (Section 3.1, angles 120/90/135 degrees, four principal-value
  triples, in units of 1e-3) and Table 3 (Section 4.2.1, four angle triples, first row of K).
  A transposed rotation, a swapped angle order or a sign error in one elementary rotation moves
  these entries far beyond the printed digits.
* ``diagnostics``: the entropy H[g] = sum_i g_i ln(g_i / W_i) of Eq. (method-entropy) has a
  closed form on an equilibrium state g_i = phi W_i P_i(u):
  H = sum_x phi ln phi + phi sum_i W_i P_i ln P_i, which is sum_x phi ln phi at u = 0
  (sum_i W_i = 1).  Mass is sum_x phi and the minimum population is phi_min W_min P_min.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def _theta(d, euler_deg):
    return torch.tensor([math.log(v) for v in d] + [math.radians(a) for a in euler_deg], dtype=torch.float64)


@pytest.mark.parametrize("row", GOLD["table1_gaussian_tensor_targets"]["rows"])
def test_tensor_from_params_reproduces_table1(row):
    """Table 1's prescribed D (printed to 4 decimals in units of 1e-3) from (ln d, ZYZ 120/90/135)."""
    D = O.tensor_from_params(_theta(row["d"], GOLD["table1_gaussian_tensor_targets"]["euler_deg"]))
    d6 = torch.stack([D[0, 0], D[0, 1], D[0, 2], D[1, 1], D[1, 2], D[2, 2]]).numpy() * 1e3
    assert np.allclose(d6, row["target_1e3"], atol=5.5e-5), d6


@pytest.mark.parametrize("row", GOLD["table3_rotated_solid"]["rows"])
def test_tensor_from_params_reproduces_table3(row):
    """Table 3's exact conductivities K_xx, K_xy, K_xz (printed to 3 decimals)."""
    K = O.tensor_from_params(_theta(row["k"], row["euler_deg"]))
    assert np.allclose(K[0].numpy(), row["K_exact"], atol=5.5e-4), K[0]


def test_tensor_from_params_per_node_batch():
    """The per-node form [6, *nodes] evaluates every node with its own parameters: the four
    Table 3 rows at once, in a 2 x 2 node layout."""
    rows = GOLD["table3_rotated_solid"]["rows"]
    th = torch.stack([_theta(r["k"], r["euler_deg"]) for r in rows], dim=1).reshape(6, 2, 2)
    K = O.tensor_from_params(th).reshape(4, 3, 3)
    for n, r in enumerate(rows):
        assert np.allclose(K[n, 0].numpy(), r["K_exact"], atol=5.5e-4)
    # symmetric positive definite with the prescribed spectrum
    ev = torch.linalg.eigvalsh(K)
    assert np.allclose(ev.numpy(), np.sort(np.array([r["k"] for r in rows]), axis=1), rtol=1e-12)


def _eq_state(phi, u):
    return O.equilibrium(torch.as_tensor(phi, dtype=torch.float64), torch.as_tensor(u, dtype=torch.float64))


def test_entropy_of_rest_equilibrium_is_phi_ln_phi():
    rng = np.random.default_rng(3)
    phi = rng.uniform(0.05, 2.0, (4, 5, 6))
    d = O.diagnostics(_eq_state(phi, (0.0, 0.0, 0.0)))
    assert d["entropy"] == pytest.approx(float(np.sum(phi * np.log(phi))), rel=1e-13)
    assert d["mass"] == pytest.approx(float(phi.sum()), rel=1e-14)
    assert d["gmin"] == pytest.approx(phi.min() / 216.0, rel=1e-14)


def test_entropy_of_moving_equilibrium():
    """u != 0: H = sum_x phi (ln phi + sum_i W_i P_i ln P_i); the second sum is evaluated here
    from the one-dimensional factors of the tensor-product weights (an independent route):
    with w(0) = 2/3, w(+-1) = 1/6 and the polynomial of Eq. (method-geq) summed over the
    3^3 product set directly, population by population, in numpy."""
    u = np.array([0.05, -0.03, 0.02])
    w1 = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
    s = 0.0
    for cx in (-1, 0, 1):
        for cy in (-1, 0, 1):
            for cz in (-1, 0, 1):
                c = np.array([cx, cy, cz], float)
                P = 1 + 3 * c @ u + 4.5 * (c @ u) ** 2 - 1.5 * u @ u
                s += w1[cx] * w1[cy] * w1[cz] * P * math.log(P)
    rng = np.random.default_rng(4)
    phi = rng.uniform(0.05, 2.0, (3, 4, 5))
    d = O.diagnostics(_eq_state(phi, u))
    assert d["entropy"] == pytest.approx(float(np.sum(phi * np.log(phi) + phi * s)), rel=1e-13)


def test_entropy_skips_non_positive_populations():
    """Populations <= 0 contribute nothing (g ln g -> 0 as g -> 0+): setting one rest-equilibrium
    population to 0 or to a negative value removes exactly its term phi W_i ln phi."""
    phi = np.full((2, 2, 3), 0.7)
    g = _eq_state(phi, (0.0, 0.0, 0.0))
    full = O.diagnostics(g)["entropy"]
    for v in (0.0, -1e-3):
        h = g.clone()
        h[5, 1, 0, 2] = v
        term = 0.7 * (1 / 54.0) * math.log(0.7)        # population 5 has two non-zero components
        assert O.diagnostics(h)["entropy"] == pytest.approx(full - term, rel=1e-13)
