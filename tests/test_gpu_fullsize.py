"""Full-size parity, in the launch configuration bench.py times: the GPU state
after K steps is read, one more step is taken, and for sampled nodes the
oracle recomputes that step node by node from the GPU's state at K (the 27
source nodes of each sampled node are collided in FP64 and streamed).

Tolerances per form: FP32 1e-6 relative L2 over the sampled populations; FP16
deviations 2e-4 and BF16 deviations 2e-3 (storage unit 4.9e-4 / 3.9e-3 on
relative deviations of order 1e-1); no sample may exceed 50x that per node.

A sample above the per-node bound is excused only where the oracle shows that one of the
collisions feeding it sits at a threshold that FP32 arithmetic can resolve either way: the
stabilizer guard <dh|dh>_H = theta^2 phi within 1 % (u != 0 only), the positivity fallback
min_i (g_i + Omega_i) within 1e-5 of the node's largest population of 0, or a far-tail node
with phi < 1e-25 (FP32 flush-to-zero and the phi > 1e-30 guard).  A sample above the bound
without such a crossing fails the test; excused samples are counted (below 1 %) and their
error is capped at max(1e-3, 50 tol): a guard crossing moves a population by kappa dh ~
theta phi.

Besides random samples, every node of four boundary lines is sampled (x = 0, x = Nx - 1,
y = 0 and z = Nz - 1), so a wrong periodic wrap or anti-bounce-back face in the staged-row
kernels shows on hundreds of samples.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import gpu_lattice

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-6, "f16dev": 2e-4, "bf16dev": 2e-3}


@pytest.fixture(scope="module")
def E():
    from paper_2605_01774_gb300 import elbm
    elbm.lib()
    return elbm


def _sample_nodes(dims, m, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    pts = np.stack([rng.integers(0, nx, m), rng.integers(0, ny, m), rng.integers(0, nz, m)], 1)
    edges = np.array([[0, 0, 0], [nx - 1, ny - 1, nz - 1], [0, ny // 2, nz - 1], [nx - 1, 0, nz // 2]])
    return np.concatenate([pts, edges, _boundary_lines(dims, seed)])


def _boundary_lines(dims, seed):
    """Every node of the lines (x = 0, y0, z0), (x = Nx - 1, y1, z1) along y, and of the lines
    y = 0 and z = Nz - 1 along x: the periodic wraps in y and z and the x faces."""
    rng = np.random.default_rng(seed + 100)
    nx, ny, nz = dims
    y0, z0, y1, z1 = (int(v) for v in rng.integers(0, min(ny, nz), 4))
    a = np.stack([np.zeros(ny, int), np.arange(ny), np.full(ny, z0)], 1)
    b = np.stack([np.full(ny, nx - 1), np.arange(ny), np.full(ny, z1)], 1)
    c = np.stack([np.arange(nx), np.zeros(nx, int), np.full(nx, y0 % nz)], 1)
    d = np.stack([np.arange(nx), np.full(nx, y1 % ny), np.full(nx, nz - 1)], 1)
    return np.concatenate([a, b, c, d])


def _threshold_nodes(g, u, S, theta):
    """Per collision: True where FP32 arithmetic can legitimately take the other branch of the
    stabilizer guard or of the positivity fallback, or where phi is in the far tail."""
    phi = g.sum(0)
    geq = O.equilibrium(phi, u)
    gneq = g - geq
    dh = gneq - O.lift(O.first_moment(gneq))
    ok = (geq > 0).all(0) & (phi > 0)
    hh = torch.where(ok, (dh * dh / torch.where(geq > 0, geq, torch.ones_like(geq))).sum(0), torch.zeros_like(phi))
    guard = torch.zeros_like(phi, dtype=torch.bool)
    if bool((u != 0).any()):
        guard = ok & ((hh / (theta * theta * torch.where(phi > 0, phi, torch.ones_like(phi))) - 1.0).abs() < 1e-2)
    post, _ = O.collide(g, u, S, theta=theta, lam_mode="reduced", fallback=False)
    scale = g.abs().max(0).values
    fb = post.min(0).values.abs() <= 1e-5 * scale
    tail = phi.abs() < 1e-25
    return guard | fb | tail


def _oracle_one_step(g_prev, dims, pts, u, S_of, theta, bc=None, src=None):
    """Pre-collision populations at pts after one step, from the pre-collision state g_prev
    (torch [27, Nz, Ny, Nx] on the GPU), recomputed node by node in FP64."""
    nx, ny, nz = dims
    C = O.C.numpy().astype(int)
    m = len(pts)
    src_nodes = np.empty((27, m, 3), dtype=np.int64)   # source node of population i of sample p
    for i in range(27):
        s = pts - C[i]
        src_nodes[i] = s
    flat = src_nodes.reshape(-1, 3)
    outside = (flat[:, 0] < 0) | (flat[:, 0] >= nx)
    fx = np.mod(flat[:, 0], nx)
    fy = np.mod(flat[:, 1], ny)
    fz = np.mod(flat[:, 2], nz)
    idx = torch.as_tensor(fx + nx * (fy + ny * fz), device=g_prev.device)
    gsrc = g_prev.reshape(27, -1)[:, idx].double().cpu()                # [27, 27*m]
    if src is not None:
        R = torch.as_tensor(src.reshape(-1)[fx + nx * (fy + ny * fz)])
        gsrc = O.source_half_step(gsrc, R, u)
    S = S_of(fx, fy, fz)
    gpost, info = O.collide(gsrc, u, S, theta=theta, lam_mode="reduced")
    excusable = _threshold_nodes(gsrc, u, S, theta).view(27, m).any(0)
    out = torch.empty(27, m, dtype=torch.float64)
    gp = gpost.view(27, 27, m)                                              # [pop, source-of-pop, sample]
    for i in range(27):
        out[i] = gp[i, i]
    if bc is not None:
        # anti-bounce-back for links entering from outside the x range
        o = torch.as_tensor(outside.reshape(27, m))
        own = torch.as_tensor(pts[:, 0] + nx * (pts[:, 1] + ny * pts[:, 2]), device=g_prev.device)
        gown = g_prev.reshape(27, -1)[:, own].double().cpu()
        if src is not None:
            Ro = torch.as_tensor(src.reshape(-1)[pts[:, 0] + nx * (pts[:, 1] + ny * pts[:, 2])])
            gown = O.source_half_step(gown, Ro, u)
        Sown = S_of(pts[:, 0], pts[:, 1], pts[:, 2])
        gpo, _ = O.collide(gown, u, Sown, theta=theta, lam_mode="reduced")
        excusable = excusable | _threshold_nodes(gown, u, Sown, theta)
        for i in range(27):
            if o[i].any():
                cx = C[i][0]
                phw = bc[0] if cx == 1 else bc[1]
                out[i, o[i]] = -gpo[O.OPP[i], o[i]] + 2.0 * O.W[i] * phw
    if src is not None:
        R = torch.as_tensor(src.reshape(-1)[pts[:, 0] + nx * (pts[:, 1] + ny * pts[:, 2])])
        out = O.source_half_step(out, R, u)
    return out, excusable


def _gpu_at(g, dims, pts):
    nx, ny, nz = dims
    idx = torch.as_tensor(pts[:, 0] + nx * (pts[:, 1] + ny * pts[:, 2]), device=g.device)
    return g.reshape(27, -1)[:, idx].double().cpu()


def _compare(name, gpu, ref, tol, excusable):
    # per-node error relative to the node's own size, with an absolute floor of 1e-6 of the
    # largest sampled node (far-tail nodes, phi down to 1e-38, are compared in absolute terms)
    nrm = torch.linalg.vector_norm(ref, dim=0)
    floor = 1e-6 * nrm.max()
    per_node = torch.linalg.vector_norm(gpu - ref, dim=0) / torch.maximum(nrm, floor)
    over = per_node > 50 * tol
    unexplained = over & ~excusable
    excused = over & excusable
    keep = ~over
    rel = (torch.linalg.vector_norm((gpu - ref)[:, keep]) / torch.linalg.vector_norm(ref[:, keep])).item()
    worst_excused = per_node[excused].max().item() if bool(excused.any()) else 0.0
    frac = excused.float().mean().item()
    print(f"{name}: sampled rel L2 {rel:.2e}, worst node within bound {per_node[keep].max().item():.2e}; "
          f"{int(over.sum())} samples above {50 * tol:.0e} ({int(unexplained.sum())} without a threshold "
          f"crossing), threshold-flagged samples {excusable.float().mean().item():.3f}, worst excused {worst_excused:.2e}")
    assert rel < tol, (name, rel)
    assert not bool(unexplained.any()), (name, int(unexplained.sum()), per_node[unexplained].max().item())
    assert frac < 0.01, (name, frac)
    assert worst_excused < max(1e-3, 50 * tol), (name, worst_excused)


@pytest.mark.parametrize("prec,background", [("f32", 0.0), ("f16dev", 0.0), ("bf16dev", 0.0), ("f32", 0.1),
                                             ("f16dev", 0.1)])
def test_plume_256_sampled(E, prec, background):
    """The bench's plume and launch.  With background > 0 a periodic mode
    background (1 + 0.5 sin(2 pi (x + 2y + 3z) / 256)) is added, so the field varies across every
    periodic seam (the plume alone leaves the faces at phi ~ e^-128, and a uniform background
    would make both sides of a seam equal): a wrong wrap in x, y or z of the staged rows then
    moves sampled boundary nodes by ~1e-3 of their size, far above the bound."""
    wl = synth.gaussian_plume(n=256)
    lat = gpu_lattice(E, wl.dims, prec, D=wl.D, u=wl.u, theta=3e-4)
    phi0 = wl.phi0 + (synth.sine_mode(wl.dims, (1, 2, 3), c0=background, amp=0.5 * background) if background else 0.0)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, dtype=torch.float32, device="cuda"))
    E.elbm_step(lat.h, 40)
    g0 = torch.empty((27,) + wl.dims[::-1], dtype=torch.float32, device="cuda")
    E.elbm_read_populations(lat.h, g0)
    E.elbm_step(lat.h, 1)
    g1 = torch.empty_like(g0)
    E.elbm_read_populations(lat.h, g1)
    torch.cuda.synchronize()
    d = E.elbm_reduce(lat.h)
    assert d["gmin"] > -1e-6
    lat.close()
    # sample where the plume lives and uniformly
    pts = np.concatenate([_sample_nodes(wl.dims, 1500, 1),
                          (np.asarray(wl.meta["mu0"]) + np.random.default_rng(2).normal(0, 10, (1500, 3))).astype(int) % 256])
    S = O.relaxation_matrix(torch.as_tensor(wl.D))
    ref, exc = _oracle_one_step(g0, wl.dims, pts, torch.as_tensor(wl.u), lambda x, y, z: S, 3e-4)
    _compare(f"plume256 {prec} background {background}", _gpu_at(g1, wl.dims, pts), ref, TOL[prec], exc)


@pytest.mark.parametrize("prec", ["f32", "f16dev"])
def test_heterogeneous_384_sampled(E, prec):
    """384^3 two-phase porous tensor field, Dirichlet x faces, Gaussian source."""
    wl = synth.heterogeneous(n=384)
    lat = gpu_lattice(E, wl.dims, prec, D6_field=wl.D6_field, bc=wl.dirichlet_x, source=wl.source, theta=3e-4)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(wl.phi0, dtype=torch.float32, device="cuda"))
    E.elbm_step(lat.h, 5)
    g0 = torch.empty((27,) + wl.dims[::-1], dtype=torch.float32, device="cuda")
    E.elbm_read_populations(lat.h, g0)
    E.elbm_step(lat.h, 1)
    g1 = torch.empty_like(g0)
    E.elbm_read_populations(lat.h, g1)
    torch.cuda.synchronize()
    lat.close()
    pts = _sample_nodes(wl.dims, 3000, 3)
    pts = np.concatenate([pts, np.array([[0, 5, 7], [383, 9, 11], [0, 383, 383], [383, 0, 0]])])
    D6f = wl.D6_field.astype(np.float32).astype(np.float64)

    def S_of(x, y, z):
        D = synth.matrix_from_d6(np.moveaxis(D6f[:, z, y, x], 0, -1))
        return O.relaxation_matrix(torch.as_tensor(D))
    src = wl.source.astype(np.float32).astype(np.float64)
    ref, exc = _oracle_one_step(g0, wl.dims, pts, torch.zeros(3, dtype=torch.float64), S_of, 3e-4,
                                bc=wl.dirichlet_x, src=src)
    _compare(f"heterogeneous384 {prec}", _gpu_at(g1, wl.dims, pts), ref, TOL[prec], exc)


def test_plume_256_long_run_deviation_forms(E):
    """300 steps of the 256^3 plume: the deviation storages stay finite past the point where
    far-tail nodes (phi ~ 1e-15, mixed-sign populations) exceed the 16-bit range, keep the
    total mass to FP32 accumulation accuracy, and track the FP32 form.  Nodes whose
    deviations do not fit are stored as their equilibrium shape and counted."""
    wl = synth.gaussian_plume(n=256)
    phi0 = torch.as_tensor(wl.phi0, dtype=torch.float32, device="cuda")
    out = {}
    for prec in ["f32", "f16dev", "bf16dev"]:
        lat = gpu_lattice(E, wl.dims, prec, D=wl.D, u=wl.u, theta=3e-4)
        E.elbm_init_equilibrium(lat.h, phi0)
        m0 = E.elbm_reduce(lat.h)["mass"]
        E.elbm_step(lat.h, 300)
        d = E.elbm_reduce(lat.h)                    # raises on non-finite populations
        proj = E.elbm_storage_projections(lat.h)
        phi = torch.empty(wl.dims[::-1], dtype=torch.float64, device="cuda")
        E.elbm_read_moments(lat.h, phi)
        lat.close()
        assert abs(d["mass"] - m0) / m0 < 1e-5, (prec, d["mass"], m0)
        out[prec] = phi
        print(f"{prec}: mass drift {abs(d['mass'] - m0) / m0:.2e}, projected node updates {proj} "
              f"({proj / (300 * phi.numel()):.2e} of all)")
        if prec == "f32":
            assert proj == 0
    ref = out["f32"]
    for prec, bound in [("f16dev", 1e-3), ("bf16dev", 1e-2)]:
        err = (torch.linalg.vector_norm(out[prec] - ref) / torch.linalg.vector_norm(ref)).item()
        print(f"{prec} vs f32 after 300 steps: rel L2 phi {err:.2e}")
        assert err < bound, (prec, err)
