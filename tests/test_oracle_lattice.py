"""Pins of the oracle's velocity set, equilibrium, lift and flux/ghost split
against the quadrature identities and closed-form moments of Sections 2.1-2.2
(P1).  Runs on CPU only."""
import json
import os
from fractions import Fraction

import pytest
import torch

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
DT = torch.float64


def test_weights_match_printed_values():
    by_m = [float(Fraction(s)) for s in GOLD["d3q27_weights"]["by_m"]]
    m = (O.C != 0).sum(1)
    for i in range(27):
        assert O.W[i].item() == pytest.approx(by_m[int(m[i])], abs=1e-16)
    # population counts per class: 1 rest, 6 axis, 12 face-diagonal, 8 corner
    assert [int((m == k).sum()) for k in range(4)] == [1, 6, 12, 8]


def test_opposite_directions():
    for i in range(27):
        assert torch.equal(O.C[O.OPP[i]], -O.C[i])
    assert O.C_INT[13] == (0, 0, 0)


def test_quadrature_identities():
    eye = torch.eye(3, dtype=DT)
    assert O.W.sum().item() == pytest.approx(1.0, abs=1e-15)
    assert torch.allclose(O.W @ O.C, torch.zeros(3, dtype=DT), atol=1e-16)
    M2 = torch.einsum("i,ia,ib->ab", O.W, O.C, O.C)
    assert torch.allclose(M2, eye / 3, atol=1e-16)
    M3 = torch.einsum("i,ia,ib,ic->abc", O.W, O.C, O.C, O.C)
    assert M3.abs().max().item() < 1e-16
    # fourth moment of the tensor-product set: (1/9)(d_ab d_cd + d_ac d_bd + d_ad d_bc)
    M4 = torch.einsum("i,ia,ib,ic,id->abcd", O.W, O.C, O.C, O.C, O.C)
    iso = (torch.einsum("ab,cd->abcd", eye, eye) + torch.einsum("ac,bd->abcd", eye, eye)
           + torch.einsum("ad,bc->abcd", eye, eye)) / 9
    assert torch.allclose(M4, iso, atol=1e-16)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_moments_closed_form(seed):
    """sum g_eq = phi, sum c g_eq = phi u, sum cc g_eq = phi (I/3 + u u),
    sum ccc g_eq = (phi/3)(u_a d_bc + u_b d_ac + u_c d_ab)."""
    g = torch.Generator().manual_seed(seed)
    phi = 0.5 + torch.rand(5, generator=g, dtype=DT)
    u = 0.1 * (torch.rand(3, 5, generator=g, dtype=DT) - 0.5)
    geq = O.equilibrium(phi, u)
    eye = torch.eye(3, dtype=DT)
    assert torch.allclose(geq.sum(0), phi, rtol=1e-15, atol=0)
    assert torch.allclose(O.first_moment(geq), phi * u, atol=1e-16)
    m2 = torch.einsum("ia,ib,in->nab", O.C, O.C, geq)
    exp2 = phi[:, None, None] * (eye / 3 + torch.einsum("an,bn->nab", u, u))
    assert torch.allclose(m2, exp2, atol=1e-15)
    m3 = torch.einsum("ia,ib,ic,in->nabc", O.C, O.C, O.C, geq)
    exp3 = (phi[:, None, None, None] / 3) * (torch.einsum("an,bc->nabc", u, eye)
                                            + torch.einsum("bn,ac->nabc", u, eye)
                                            + torch.einsum("cn,ab->nabc", u, eye))
    assert torch.allclose(m3, exp3, atol=1e-15)


def test_lift_identities():
    a = torch.tensor([0.3, -0.7, 1.1], dtype=DT)
    p = O.lift(a)
    assert abs(p.sum().item()) < 1e-16
    assert torch.allclose(O.C.T @ p, a, atol=1e-15)
    # only non-zero low-order moment is the first: second moment vanishes
    assert torch.einsum("ia,ib,i->ab", O.C, O.C, p).abs().max().item() < 1e-16


def test_flux_ghost_split_identities():
    g0 = torch.Generator().manual_seed(3)
    g = 0.01 + torch.rand(27, 7, generator=g0, dtype=DT)
    u = torch.tensor([0.05, -0.03, 0.02], dtype=DT)
    phi = O.zeroth_moment(g)
    geq = O.equilibrium(phi, u)
    j = O.first_moment(g - geq)
    ds = O.lift(j)
    dh = g - geq - ds
    tol = 1e-15 * phi.max().item()          # rounding of sums of 27 terms of size ~phi/27
    assert dh.sum(0).abs().max().item() < 4 * tol
    assert ds.sum(0).abs().max().item() < 4 * tol
    assert O.first_moment(dh).abs().max().item() < 4 * tol
    assert torch.allclose(O.first_moment(ds), j, atol=4 * tol)
    # j = sum c g - phi u (Eq. method-first-moment)
    assert torch.allclose(j, O.first_moment(g) - phi * u[:, None], atol=4 * tol)
