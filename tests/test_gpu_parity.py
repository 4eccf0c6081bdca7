"""GPU (C ABI) vs FP64 oracle parity on seeded inputs.

Tolerances: FP64 1e-12 relative L2 (the scheme's target).  FP32 and the
16-bit deviation storages: bounds derived from the storage rounding unit
(FP32 6e-8, FP16 4.9e-4, BF16 3.9e-3 on relative deviations of a few 1e-2)
accumulated over the steps; each test states its bound."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import gpu_lattice, oracle_problem, read_phi, read_pops, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2605_01774_gb300 import elbm
    elbm.lib()
    return elbm


def test_config1_decay_fp64(E):
    """32^3 periodic, u = 0, rotated D = R diag(0.05, 0.005, 0.0005) R^T, 200 steps, FP64."""
    wl = synth.decay_mode(n=32, seed=1, steps=200)
    lat = gpu_lattice(E, wl.dims, "f64", D=wl.D)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(wl.phi0, device="cuda"))
    E.elbm_step(lat.h, 200)
    g = read_pops(E, lat)
    prob = oracle_problem(D=wl.D, theta=1e-8, lam_mode="literal")
    ref = O.run(O.init_equilibrium(wl.phi0, wl.u), prob, 200)
    err_g = rel_l2(g, ref)
    err_phi = rel_l2(g.sum(0), ref.sum(0))
    print(f"config1 fp64: rel L2 pops {err_g:.2e} phi {err_phi:.2e}")
    assert err_g < 1e-12 and err_phi < 1e-12
    d = E.elbm_reduce(lat.h)
    assert d["n_fallback"] == 0
    assert abs(d["mass"] - wl.phi0.sum()) / wl.phi0.sum() < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 5, 7), (7, 1, 2)])
@pytest.mark.parametrize("bc", [None, (1.3, 0.7)])
def test_brute_force_tiny_fp64(E, dims, bc):
    """Random positive states, u != 0, per-node tensor field, source, 3 steps: node-by-node 1e-13."""
    rng = synth.rng(sum(dims))
    N = int(np.prod(dims))
    g0 = (O.W.numpy()[:, None] * (1 + 0.3 * rng.standard_normal((27, N)))).clip(1e-3)
    g0 = g0.reshape((27,) + dims[::-1])
    D6 = np.empty((6,) + dims[::-1])
    for idx in np.ndindex(*dims[::-1]):
        R = synth.rot_zyz(*synth.haar_euler(rng))
        D6[(slice(None),) + idx] = synth.d6_from_matrix(synth.tensor_from_principal(10 ** rng.uniform(-4, -1, 3), R))
    u = (0.04, -0.02, 0.03)
    src = 1e-3 * rng.uniform(0, 1, dims[::-1])
    lat = gpu_lattice(E, dims, "f64", D6_field=D6, u=u, bc=bc, source=src)
    E.elbm_write_populations(lat.h, torch.as_tensor(g0, device="cuda"))
    back = read_pops(E, lat)
    assert rel_l2(back, g0) < 1e-15
    prob = oracle_problem(S_field_D=D6.astype(np.float32).astype(np.float64), u=u, bc=bc, source=src,
                          theta=1e-8, lam_mode="literal")
    ref = torch.as_tensor(g0)
    for n in range(3):
        E.elbm_step(lat.h, 1)
        ref = O.step(ref, prob, n)
        g = read_pops(E, lat)
        diff = (g - ref).abs().max().item() / ref.abs().max().item()
        assert diff < 1e-13, (n, diff)


@pytest.mark.parametrize("prec,bound", [("f32", 2e-6), ("f16dev", 3e-4), ("bf16dev", 3e-3)])
def test_gaussian_reduced_precision(E, prec, bound):
    """24^3 advected anisotropic plume (u != 0, anisotropy 1e4), 40 steps, vs the FP64 oracle with
    the same guard theta; bound on rel L2 of phi."""
    wl = synth.gaussian_plume(n=24, sigma0=4.0, eig=(0.1, 1e-3, 1e-5), steps=40)
    lat = gpu_lattice(E, wl.dims, prec, D=wl.D, u=wl.u)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(wl.phi0, device="cuda"))
    E.elbm_step(lat.h, 40)
    phi = read_phi(E, lat)
    prob = oracle_problem(D=wl.D, u=wl.u, theta=3e-4)
    ref = O.run(O.init_equilibrium(wl.phi0, wl.u), prob, 40).sum(0)
    err = rel_l2(phi, ref)
    linf = (phi - ref).abs().max().item() / ref.abs().max().item()
    print(f"gaussian {prec}: rel L2 phi {err:.2e}, Linf {linf:.2e}")
    assert err < bound


@pytest.mark.parametrize("prec", ["f64", "f32", "f16dev", "bf16dev"])
def test_mass_and_checkpoint(E, prec):
    wl = synth.gaussian_plume(n=16, sigma0=3.0, eig=(0.05, 0.01, 0.002), steps=10)
    phi0 = 0.5 + wl.phi0
    lat = gpu_lattice(E, wl.dims, prec, D=wl.D, u=wl.u)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    m0 = E.elbm_reduce(lat.h)["mass"]
    E.elbm_step(lat.h, 5)
    nb = E.elbm_checkpoint_size(lat.h)
    buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
    E.elbm_checkpoint_save(lat.h, buf)
    E.elbm_step(lat.h, 5)
    a = read_pops(E, lat)
    E.elbm_checkpoint_load(lat.h, buf)
    assert E.elbm_get_step(lat.h) == 5
    E.elbm_step(lat.h, 5)
    b = read_pops(E, lat)
    assert torch.equal(a, b)
    m1 = E.elbm_reduce(lat.h)["mass"]
    tol = {"f64": 1e-14, "f32": 1e-6, "f16dev": 1e-6, "bf16dev": 1e-6}[prec]
    assert abs(m1 - m0) / m0 < tol, (prec, abs(m1 - m0) / m0)


def test_reduce_matches_oracle_diagnostics(E):
    wl = synth.gaussian_plume(n=12, sigma0=3.0, eig=(0.05, 0.01, 0.002), steps=4)
    lat = gpu_lattice(E, wl.dims, "f64", D=wl.D, u=wl.u)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(wl.phi0, device="cuda"))
    E.elbm_step(lat.h, 4)
    d = E.elbm_reduce(lat.h)
    g = read_pops(E, lat)
    ref = O.diagnostics(g)
    assert d["mass"] == pytest.approx(ref["mass"], rel=1e-13)
    assert d["entropy"] == pytest.approx(ref["entropy"], rel=1e-12)
    assert d["gmin"] == pytest.approx(ref["gmin"], rel=1e-12, abs=1e-300)


def test_fallback_parity_fp64(E):
    """Adversarial step function (weak diffusivities 1e-6, u = 0.1): identical fallback counts."""
    n = 12
    phi0 = np.where(np.arange(n)[None, None, :] < n // 2, 1.0, 1e-3) * np.ones((n, n, n))
    u = (0.1, 0.0, 0.0)
    D = np.diag([1e-6, 1e-6, 0.2])
    lat = gpu_lattice(E, (n, n, n), "f64", D=D, u=u)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    prob = oracle_problem(D=D, u=u, theta=1e-8, lam_mode="literal")
    ref = O.init_equilibrium(phi0, u)
    for k in range(10):
        ref = O.step(ref, prob, k)
    E.elbm_step(lat.h, 10)
    g = read_pops(E, lat)
    d = E.elbm_reduce(lat.h)
    print("fallback nodes gpu", d["n_fallback"], "oracle", prob.stats["fallback_nodes"])
    assert d["n_fallback"] == prob.stats["fallback_nodes"] > 0
    assert rel_l2(g, ref) < 1e-12
    assert d["gmin"] >= -1e-17


def test_heterogeneous_dirichlet_source_fp32(E):
    """Two-phase porous tensor field, smooth rotation field, Gaussian source, Dirichlet x, 20 steps."""
    wl = synth.heterogeneous(dims=(20, 12, 10), src_amp=1e-3, src_width=3.0)
    for prec, bound in (("f64", 1e-12), ("f32", 1e-6), ("f16dev", 2e-4)):
        lat = gpu_lattice(E, wl.dims, prec, D6_field=wl.D6_field, bc=wl.dirichlet_x, source=wl.source)
        E.elbm_init_equilibrium(lat.h, torch.as_tensor(wl.phi0, device="cuda"))
        E.elbm_step(lat.h, 20)
        phi = read_phi(E, lat)
        prob = oracle_problem(S_field_D=wl.D6_field.astype(np.float32).astype(np.float64), bc=wl.dirichlet_x,
                              source=wl.source, theta=1e-8)
        ref = O.run(O.init_equilibrium(wl.phi0, wl.u), prob, 20).sum(0)
        err = rel_l2(phi, ref)
        print(f"heterogeneous {prec}: rel L2 phi {err:.2e}")
        assert err < bound, (prec, err)


def test_params_field_matches_oracle_parametrisation(E):
    p = synth.adjoint_problem(n=10, steps=6, obs=(3, 6))
    th = p["theta0"].astype(np.float32)
    lat = gpu_lattice(E, p["dims"], "f64", params_field=th, u=p["u"])
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(p["phi0"], device="cuda"))
    E.elbm_step(lat.h, 6)
    g = read_pops(E, lat)
    D = O.tensor_from_params(torch.as_tensor(th.astype(np.float64)))
    prob = O.Problem(u=torch.as_tensor(p["u"]), S=O.relaxation_matrix(D), theta=1e-8)
    ref = O.run(O.init_equilibrium(p["phi0"], p["u"]), prob, 6)
    # T field is stored in FP32 (relative rounding 6e-8 of the relaxation complement)
    assert rel_l2(g, ref) < 1e-9


def test_flux_readout(E):
    """q = j - S j / 2: at the exact steady state of linear conduction q = D_{.x} G."""
    K = synth.tensor_from_principal((100, 10, 0.01), synth.rot_zyz_deg(135, 35, 75)) * 1e-3
    dims = (8, 2, 2)
    lat = gpu_lattice(E, dims, "f64", D=K, bc=(2.0, 1.0))
    prob = oracle_problem(D=K, bc=(2.0, 1.0), fallback=False)
    # exact fixed point from the oracle's affine map, loaded through write_populations
    from test_oracle_boundary import _fixed_point
    gfix = _fixed_point(prob, dims)
    E.elbm_write_populations(lat.h, gfix.to("cuda"))
    E.elbm_step(lat.h, 3)
    phi = torch.empty(dims[::-1], dtype=torch.float64, device="cuda")
    q = torch.empty((3,) + dims[::-1], dtype=torch.float64, device="cuda")
    E.elbm_read_moments(lat.h, phi, q)
    torch.cuda.synchronize()
    x = np.arange(8)
    assert np.abs(phi.cpu().numpy() - (2.0 - (x + 0.5) / 8)).max() < 1e-12
    assert np.allclose(q.cpu().numpy() * 8, K[:, 0][:, None, None, None], rtol=1e-11, atol=1e-16)


def test_error_paths(E):
    lat = E.Lattice((8, 8, 8), "f32")
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_step(lat.h, 1)
    assert ei.value.status == 8                      # no state yet
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_set_tensor_uniform(lat.h, [1.0, 2.0, 0, 1.0, 0, 1.0])
    assert ei.value.status == 2
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_set_velocity_uniform(lat.h, [0.9, 0, 0])
    assert ei.value.status == 3
    bad = torch.zeros(6, 512, dtype=torch.float32, device="cuda")
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_set_tensor_field(lat.h, bad)
    assert ei.value.status == 2
    E.elbm_set_tensor_uniform(lat.h, [0.1, 0, 0, 0.1, 0, 0.1])
    phi = torch.ones(512, dtype=torch.float32, device="cuda")
    E.elbm_init_equilibrium(lat.h, phi)
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_set_velocity_uniform(lat.h, [0.01, 0, 0])
    assert ei.value.status == 8
    g = torch.full((27, 512), float("nan"), dtype=torch.float32, device="cuda")
    E.elbm_write_populations(lat.h, g)
    d = E.elbm_reduce(lat.h, allow_nonfinite=True)
    assert d["status"] == 6


def test_host_buffers_roundtrip(E):
    """Host (numpy) inputs and outputs through the same calls."""
    wl = synth.decay_mode(n=8, seed=2, steps=3)
    lat = gpu_lattice(E, wl.dims, "f32", D=wl.D)
    E.elbm_init_equilibrium(lat.h, wl.phi0.astype(np.float32))
    E.elbm_step(lat.h, 3)
    out = np.empty(wl.dims[::-1], dtype=np.float32)
    E.elbm_read_moments(lat.h, out)
    dev = read_phi(E, lat).numpy()
    assert np.allclose(out, dev, rtol=1e-7)


def test_time_dependent_source_schedule_fp64(E):
    """Source R(x, t) = a(t) f(x) evaluated at mid-step times (Section 3.3), per-node tensor,
    u != 0: amplitude schedule through elbm_step_source_schedule vs the oracle's callable source."""
    import synth.source_benchmark as SB
    p = SB.setup(n=12, d=(1e-2, 1e-3, 1e-6), t_end=40 / 144.0)
    steps = p["steps"]
    lat = gpu_lattice(E, p["dims"], "f64", D6_field=p["D6"], u=p["u_lat"], source=p["f"])
    E.elbm_set_source_amplitude(lat.h, p["amp"][0])
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(p["psi0"], device="cuda"))
    E.elbm_step_source_schedule(lat.h, p["amp"])
    g = read_pops(E, lat)
    f32 = torch.as_tensor(p["f"].astype(np.float32).astype(np.float64))
    dt, A = p["dt"], p["A"]
    prob = oracle_problem(S_field_D=p["D6"].astype(np.float32).astype(np.float64), u=p["u_lat"], theta=1e-8,
                          lam_mode="literal")
    prob.source = lambda tmid: dt * np.exp(A * tmid * dt) * f32
    ref = O.run(O.init_equilibrium(p["psi0"], p["u_lat"]), prob, steps)
    err = rel_l2(g, ref)
    print(f"time-dependent source fp64: rel L2 pops {err:.2e} over {steps} steps")
    assert err < 1e-12


@pytest.mark.parametrize("prec,bound", [("f64", 1e-11), ("f32", 2e-6)])
def test_exact_entropy_root_mode(E, prec, bound):
    """lambda from the exact root of Eq. (method-entropy-root) (FP64 Newton on the GPU for every
    precision) vs the oracle's brentq root, 10^3 plume with u != 0, 6 steps."""
    wl = synth.gaussian_plume(n=10, sigma0=2.5, eig=(0.05, 0.01, 0.002), steps=6)
    phi0 = 0.3 + wl.phi0
    theta = 1e-8 if prec == "f64" else 3e-4          # each precision's guard, on both sides
    lat = gpu_lattice(E, wl.dims, prec, D=wl.D, u=wl.u, theta=theta)
    E.elbm_set_lambda_mode(lat.h, 1)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    E.elbm_step(lat.h, 6)
    g = read_pops(E, lat)
    prob = oracle_problem(D=wl.D, u=wl.u, theta=theta, lam_mode="root")
    ref = O.run(O.init_equilibrium(phi0, wl.u), prob, 6)
    prob_cf = oracle_problem(D=wl.D, u=wl.u, theta=theta, lam_mode="literal")
    ref_cf = O.run(O.init_equilibrium(phi0, wl.u), prob_cf, 6)
    err = rel_l2(g, ref)
    print(f"root mode {prec}: rel L2 vs oracle root {err:.2e}; root vs closed form {rel_l2(ref, ref_cf):.2e}")
    assert err < bound
    assert rel_l2(ref, ref_cf) > 10 * bound or prec == "f32"


@pytest.mark.parametrize("prec,bound", [("f64", 1e-12), ("f32", 1e-6), ("f16dev", 2e-4)])
def test_velocity_field(E, prec, bound):
    """Per-node velocity u(x) (some nodes exactly 0), rotated tensor, 6 steps: populations and
    the flux read-out q = j - S j / 2 against the oracle with the same field."""
    dims = (10, 8, 6)
    rng = synth.rng(31)
    x, y, z = synth.grid(dims)
    u = np.stack([0.04 * np.sin(2 * np.pi * y / 8), 0.03 * np.cos(2 * np.pi * z / 6), 0.02 * np.sin(2 * np.pi * x / 10)])
    u[:, 0, 0, :] = 0.0
    u = u.astype(np.float32).astype(np.float64)
    D = synth.tensor_from_principal((0.05, 0.01, 0.002), synth.rot_zyz(*synth.haar_euler(rng)))
    phi0 = 1.0 + 0.3 * synth.gaussian(dims, (4.5, 3.5, 2.5), 2.0)
    lat = gpu_lattice(E, dims, prec, D=D, theta=1e-8 if prec == "f64" else 3e-4)
    E.elbm_set_velocity_field(lat.h, torch.as_tensor(u, dtype=torch.float32, device="cuda"))
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    E.elbm_step(lat.h, 6)
    g = read_pops(E, lat)
    phi = torch.empty(dims[::-1], dtype=torch.float64, device="cuda")
    q = torch.empty((3,) + dims[::-1], dtype=torch.float64, device="cuda")
    E.elbm_read_moments(lat.h, phi, q)
    torch.cuda.synchronize()
    ut = torch.as_tensor(u)
    prob = O.Problem(u=ut, S=O.relaxation_matrix(torch.as_tensor(D)), theta=1e-8 if prec == "f64" else 3e-4)
    ref = O.run(O.init_equilibrium(phi0, ut), prob, 6)
    qref = O.flux_q(ref, ut, prob.S)
    err, qerr = rel_l2(g, ref), rel_l2(q.cpu(), qref)
    print(f"velocity field {prec}: rel L2 pops {err:.2e}, flux {qerr:.2e}")
    assert err < bound
    assert qerr < max(bound, 1e-9) * 1e3
    # invalid fields are rejected
    bad = torch.zeros((3,) + dims[::-1], dtype=torch.float32, device="cuda")
    bad[0, 0, 0, 0] = 0.9
    lat2 = E.Lattice(dims, prec)
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_set_velocity_field(lat2.h, bad)
    assert ei.value.status == 3


def test_fp32_exact_mass_option(E):
    """FP32 storage: with the default exact stored mass the total mass of the advected plume
    stays to ~1e-9 over 200 steps; switched off, the rounding of the updates drifts it by
    orders of magnitude more.  Both stay within FP32 parity of each other."""
    wl = synth.gaussian_plume(n=64, sigma0=6.0, eig=(0.05, 0.005, 1e-5), steps=200)
    out = {}
    for on in (1, 0):
        lat = gpu_lattice(E, wl.dims, "f32", D=wl.D, u=wl.u)
        E.elbm_set_exact_mass(lat.h, on)
        E.elbm_init_equilibrium(lat.h, torch.as_tensor(wl.phi0, device="cuda"))
        m0 = E.elbm_reduce(lat.h)["mass"]
        E.elbm_step(lat.h, 200)
        out[on] = (abs(E.elbm_reduce(lat.h)["mass"] - m0) / m0, read_phi(E, lat))
        lat.close()
    print(f"FP32 mass drift over 200 steps: exact {out[1][0]:.2e}, plain {out[0][0]:.2e}")
    assert out[1][0] < 1e-7
    assert out[1][0] < out[0][0]
    assert rel_l2(out[1][1], out[0][1]) < 1e-4
    with pytest.raises(E.ElbmError):
        E.elbm_set_exact_mass(E.Lattice((8, 8, 8), "f32").h, 2)
