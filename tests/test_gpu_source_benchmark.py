"""The source-driven variable-tensor benchmark of Section 3.3 at the paper's size:
128^3 on [0,1)^3, u = (1,1,1) (lattice 1/128), Pe = 1e6, K = diag(d1 (2 - S), d2, d3),
49 152 steps to t = 3, shifted scalar psi = phi + 2 (the paper leaves the shift open).

The FP64 GPU path reproduces the printed global relative errors (6.154e-4 and
6.220e-4) to their printed digits, the L2 / Linf errors inside the printed ranges
and the mass drift below the printed bound.  FP32 is reported: its relative error
on this run is larger (per-step increments of 1e-5 of the state)."""
import json
import os

import numpy as np
import pytest
import torch

import synth.source_benchmark as SB

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))["section33_source_driven"]


@pytest.fixture(scope="module")
def E():
    from paper_2605_01774_gb300 import elbm
    elbm.lib()
    return elbm


def _run(E, prec, d, theta, n=128, shift=2.0):
    p = SB.setup(n=n, d=tuple(d), shift=shift)
    lat = E.Lattice(p["dims"], prec)
    E.elbm_set_tensor_field(lat.h, torch.as_tensor(p["D6"], dtype=torch.float32, device="cuda"))
    E.elbm_set_velocity_uniform(lat.h, p["u_lat"])
    E.elbm_set_source(lat.h, torch.as_tensor(p["f"], dtype=torch.float32, device="cuda"))
    E.elbm_set_params(lat.h, theta=theta)
    E.elbm_set_source_amplitude(lat.h, p["amp"][0])
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(p["psi0"], device="cuda"))
    E.elbm_step_source_schedule(lat.h, p["amp"])
    phi = torch.empty(p["dims"][::-1], dtype=torch.float64, device="cuda")
    E.elbm_read_moments(lat.h, phi)
    torch.cuda.synchronize()
    d = E.elbm_reduce(lat.h)
    lat.close()
    num = phi.cpu().numpy() - shift
    ex = p["exact"](GOLD["t_end"])
    # mass of phi: initial sum plus what the (FP32-stored) source injects, sum_x R(x) sum_n a_n
    expected = p["S"].sum() + p["f"].astype(np.float32).astype(np.float64).sum() * p["amp"].sum()
    return dict(gre=float(np.linalg.norm(num - ex) / np.linalg.norm(ex)),
                l2=float(np.sqrt(((num - ex) ** 2).mean())), linf=float(np.abs(num - ex).max()),
                # physical mass on [0,1)^3: integral of phi = sum(phi) dx^3
                mass=float((num.sum() - expected) / n ** 3), fallback=d["n_fallback"])


@pytest.mark.parametrize("case", [0, 3])
def test_section33_fp64_reproduces_printed_errors(E, case):
    c = GOLD["cases"][case]
    r = _run(E, "f64", c["d"], 1e-8)
    print(f"d = {c['d']}: GRE {r['gre']:.5e} (paper {c['gre']:.4e}), L2 {r['l2']:.4e}, Linf {r['linf']:.4e}, "
          f"mass {r['mass']:.2e}")
    assert r["fallback"] == 0
    assert abs(r["gre"] - c["gre"]) < 1e-7                     # printed to 4 digits
    lo, hi = GOLD["l2_range"]
    assert lo - 5e-7 <= r["l2"] <= hi + 5e-7
    assert r["linf"] < GOLD["linf_max"]
    assert abs(r["mass"]) < GOLD["mass_drift_max"]


def test_section33_fp32_error_is_reported(E):
    c = GOLD["cases"][3]
    r = _run(E, "f32", c["d"], 3e-4)
    print(f"FP32 d = {c['d']}: GRE {r['gre']:.4e} (FP64 / paper {c['gre']:.4e}), mass {r['mass']:.2e}")
    assert r["gre"] < 5e-3
