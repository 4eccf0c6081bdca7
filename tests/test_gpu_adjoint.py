"""Hand-written adjoint of the step (per-node tensor parameters) against the
FP64 CPU reference (torch reverse mode over the oracle) and against central
finite differences of the GPU forward."""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.adjoint as OA
import synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def E():
    from paper_2605_01774_gb300 import elbm
    elbm.lib()
    return elbm


def _small(n=10, seed=5):
    p = synth.adjoint_problem(n=n, seed=seed, steps=30, obs=(15, 30))
    return p


def _rand_state(p, seed):
    rng = np.random.default_rng(seed)
    u = torch.as_tensor(p["u"])
    geq = O.init_equilibrium(p["phi0"], u)
    return geq * (1 + 0.05 * torch.as_tensor(rng.standard_normal(geq.shape)))


def test_forward_step_matches_oracle(E):
    p = _small()
    h = E.elbm_adjoint_create(p["dims"], "f64")
    E.elbm_adjoint_configure(h, p["u"], 1e-8, 7)
    g = _rand_state(p, 1)
    th = torch.as_tensor(p["theta0"])
    out = torch.empty_like(g, device=DEV)
    E.elbm_adjoint_step(h, th.to(DEV), g.to(DEV), g_next=out)
    S = O.relaxation_matrix(O.tensor_from_params(th))
    ref = O.step(g, O.Problem(u=torch.as_tensor(p["u"]), S=S, theta=1e-8), 0)
    assert ((out.cpu() - ref).abs().max() / ref.abs().max()).item() < 1e-13
    E.elbm_adjoint_destroy(h)


def test_one_step_vjp_matches_reverse_mode(E):
    """(dG'/dG)^T y and (dG'/dtheta)^T y against torch reverse mode through the oracle."""
    p = _small()
    h = E.elbm_adjoint_create(p["dims"], "f64")
    E.elbm_adjoint_configure(h, p["u"], 1e-8, 7)
    g = _rand_state(p, 2)
    th = torch.as_tensor(p["theta0"])
    ybar = torch.as_tensor(np.random.default_rng(3).standard_normal(g.shape))
    gbar = torch.empty_like(g, device=DEV)
    grad = torch.empty_like(th, device=DEV)
    E.elbm_adjoint_step(h, th.to(DEV), g.to(DEV), gbar_next=ybar.to(DEV), gbar=gbar, grad6=grad)
    gg = g.clone().requires_grad_(True)
    tt = th.clone().requires_grad_(True)
    S = O.relaxation_matrix(O.tensor_from_params(tt))
    out = O.step(gg, O.Problem(u=torch.as_tensor(p["u"]), S=S, theta=1e-8), 0)
    rg, rt = torch.autograd.grad((out * ybar).sum(), (gg, tt))
    e1 = (torch.linalg.vector_norm(gbar.cpu() - rg) / torch.linalg.vector_norm(rg)).item()
    e2 = (torch.linalg.vector_norm(grad.cpu() - rt) / torch.linalg.vector_norm(rt)).item()
    print(f"one-step VJP rel err: populations {e1:.2e}, parameters {e2:.2e}")
    assert e1 < 1e-11 and e2 < 1e-10
    # dot-product test against central differences of the GPU forward
    v = torch.as_tensor(np.random.default_rng(4).standard_normal(g.shape)) * 1e-3
    hh = 1e-6
    fp = torch.empty_like(g, device=DEV)
    fm = torch.empty_like(g, device=DEV)
    E.elbm_adjoint_step(h, th.to(DEV), (g + hh * v).to(DEV), g_next=fp)
    E.elbm_adjoint_step(h, th.to(DEV), (g - hh * v).to(DEV), g_next=fm)
    lhs = (ybar * ((fp - fm).cpu() / (2 * hh))).sum().item()
    rhs = (gbar.cpu() * v).sum().item()
    assert abs(lhs - rhs) / abs(rhs) < 1e-7
    E.elbm_adjoint_destroy(h)


def test_misfit_gradient_matches_fp64_cpu_adjoint(E):
    """10^3, 30 steps, observations at 15 and 30, checkpoints every 7 steps (segments that do
    not divide the run): J and dJ/dtheta against torch reverse mode through the oracle."""
    p = _small()
    targets = OA.forward_snapshots(p["theta_true"], p["phi0"], p["u"], 30, (15, 30))
    J_ref, g_ref, nfb = OA.misfit_gradient(p["theta0"], p["phi0"], p["u"], 30, (15, 30), targets)
    assert nfb == 0
    h = E.elbm_adjoint_create(p["dims"], "f64")
    E.elbm_adjoint_configure(h, p["u"], 1e-8, 7)
    tg = torch.stack([targets[15], targets[30]]).to(DEV).contiguous()
    grad = torch.empty(p["theta0"].shape, dtype=torch.float64, device=DEV)
    J, nfb = E.elbm_adjoint_misfit(h, torch.as_tensor(p["theta0"], device=DEV), torch.as_tensor(p["phi0"], device=DEV),
                                   30, [15, 30], tg, grad6=grad)
    assert nfb == 0
    assert J == pytest.approx(J_ref, rel=1e-11)
    err = (torch.linalg.vector_norm(grad.cpu() - g_ref) / torch.linalg.vector_norm(g_ref)).item()
    print(f"misfit gradient vs FP64 CPU adjoint: rel err {err:.2e}")
    assert err < 1e-9
    # through the autograd Function
    F = E.tensor_misfit_function()
    th = torch.as_tensor(p["theta0"], device=DEV).requires_grad_(True)
    Jt = F.apply(th, h, torch.as_tensor(p["phi0"], device=DEV), 30, [15, 30], tg)
    Jt.backward()
    assert torch.allclose(th.grad, grad, rtol=1e-14, atol=0)
    # without a gradient to compute (no_grad, or theta not requiring one) only the forward sweep
    # runs; J is the same and the result carries no graph
    with torch.no_grad():
        Jn = F.apply(th, h, torch.as_tensor(p["phi0"], device=DEV), 30, [15, 30], tg)
    Jd = F.apply(th.detach(), h, torch.as_tensor(p["phi0"], device=DEV), 30, [15, 30], tg)
    assert Jn.item() == Jt.item() and Jd.item() == Jt.item()
    assert not Jn.requires_grad and not Jd.requires_grad
    E.elbm_adjoint_destroy(h)


def test_config5_gradient_vs_central_differences(E):
    """64^3, u = (0.02, 0, 0), 500 steps, observations at 250 and 500, checkpoints every 50;
    FP64 adjoint vs central differences (h = 1e-6) on 20 seeded (node, component) pairs."""
    p = synth.adjoint_problem()
    dims, n = p["dims"], 64
    h = E.elbm_adjoint_create(dims, "f64")
    E.elbm_adjoint_configure(h, p["u"], 1e-8, 50)
    th_true = torch.as_tensor(p["theta_true"], device=DEV)
    phi0 = torch.as_tensor(p["phi0"], device=DEV)
    # synthetic observations from the true parameters (GPU forward)
    N = n ** 3
    g = (phi0.reshape(1, -1) * torch.as_tensor(
        [float(w) * (1 + 3 * c @ p["u"] + 4.5 * (c @ p["u"]) ** 2 - 1.5 * p["u"] @ p["u"])
         for w, c in zip(O.W.numpy(), O.C.numpy())], device=DEV).reshape(27, 1)).contiguous()
    nxt = torch.empty_like(g)
    snaps = {}
    for t in range(500):
        E.elbm_adjoint_step(h, th_true, g, g_next=nxt)
        g, nxt = nxt, g
        if t + 1 in (250, 500):
            snaps[t + 1] = g.sum(0)
    tg = torch.stack([snaps[250], snaps[500]]).contiguous()
    th0 = torch.as_tensor(p["theta0"], device=DEV).contiguous()
    grad = torch.empty_like(th0)
    J0, nfb = E.elbm_adjoint_misfit(h, th0, phi0, 500, [250, 500], tg, grad6=grad)
    assert nfb == 0 and J0 > 0
    # 20 seeded (node, component) pairs where the misfit is sensitive: nodes within 8 of the
    # plume centre (far nodes have gradients of 1e-13, below the FD noise floor of ~1e-10)
    rng = np.random.default_rng(55)
    hstep = 1e-5
    worst = 0.0
    for _ in range(20):
        comp = int(rng.integers(0, 6))
        x, y, z = (31.5 + rng.uniform(-8, 8, 3)).astype(int)
        node = int(x + n * (y + n * z))
        tp = th0.clone()
        tp.view(6, -1)[comp, node] += hstep
        tm = th0.clone()
        tm.view(6, -1)[comp, node] -= hstep
        Jp, _ = E.elbm_adjoint_misfit(h, tp, phi0, 500, [250, 500], tg)
        Jm, _ = E.elbm_adjoint_misfit(h, tm, phi0, 500, [250, 500], tg)
        fd = (Jp - Jm) / (2 * hstep)
        ad = grad.view(6, -1)[comp, node].item()
        rel = abs(ad - fd) / max(abs(fd), 1e-300)
        worst = max(worst, rel)
        print(f"theta[{comp}, {node}]: adjoint {ad:.9e} central FD {fd:.9e} rel {rel:.2e}")
    assert worst < 1e-4
    # FP32 adjoint against the FP64 one, both with the FP32 guard theta = 3e-4
    E.elbm_adjoint_configure(h, p["u"], 3e-4, 50)
    J64, _ = E.elbm_adjoint_misfit(h, th0, phi0, 500, [250, 500], tg, grad6=grad)
    h32 = E.elbm_adjoint_create(dims, "f32")
    E.elbm_adjoint_configure(h32, p["u"], 3e-4, 50)
    g32 = torch.empty(th0.shape, dtype=torch.float32, device=DEV)
    J32, nfb32 = E.elbm_adjoint_misfit(h32, th0.float(), phi0.float(), 500, [250, 500], tg.float(), grad6=g32)
    e = (torch.linalg.vector_norm(g32.double() - grad) / torch.linalg.vector_norm(grad)).item()
    print(f"FP32 vs FP64 adjoint: J rel {abs(J32 - J64) / J64:.2e}, gradient rel L2 {e:.2e}")
    assert nfb32 == 0
    assert e < 5e-2
    E.elbm_adjoint_destroy(h32)
    E.elbm_adjoint_destroy(h)
