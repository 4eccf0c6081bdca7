"""D2Q9 step (include/elbm2d.h) against the D2Q9 oracle, through the C ABI.

FP64: node by node to 1e-12 of the largest population, on lattices that span several blocks
with a ragged tail along x (300 nodes per row), narrow rows that run two-dimensional blocks,
uniform and per-node tensors and velocities (Section 4.1 runs D2Q9 with y-dependent K and
u), the entropic amplitude active, and the positivity fallback taken (identical counts).
FP32: relative L2 bound derived from the FP32 unit (6e-8 per operation, ~40 operations per
population per step, accumulated over the steps).  At the size the bench times, one step is
checked on sampled nodes (plus every node of the four boundary rows) against the oracle's
collision of each sample's 3 x 3 source patch."""
import math

import numpy as np
import pytest
import torch

import oracle.d2q9 as O2
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2605_01774_gb300 import elbm
    elbm.lib()
    return elbm


def _rot2(a):
    return np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])


def _fields(nx, ny, seed):
    """Channel-like fields of Section 4.1's shape on a periodic box (synth.channel2d)."""
    return synth.channel2d(nx, ny, seed)


def _S_field(D3):
    D = np.empty(D3.shape[1:] + (2, 2))
    D[..., 0, 0], D[..., 0, 1], D[..., 1, 0], D[..., 1, 1] = D3[0], D3[1], D3[1], D3[2]
    return O2.relaxation_matrix(torch.as_tensor(D))


def _lattice(E, dims, prec, u=None, D=None, ufield=None, D3=None, theta=None, fallback=True):
    lat = E.Lattice2D(dims, prec)
    if D is not None:
        E.elbm2d_set_tensor_uniform(lat.h, [D[0, 0], D[0, 1], D[1, 1]])
    if D3 is not None:
        E.elbm2d_set_tensor_field(lat.h, torch.as_tensor(D3, dtype=torch.float32, device="cuda"))
    if ufield is not None:
        E.elbm2d_set_velocity_field(lat.h, torch.as_tensor(ufield, dtype=torch.float32, device="cuda"))
    elif u is not None:
        E.elbm2d_set_velocity_uniform(lat.h, u)
    E.elbm2d_set_params(lat.h, theta=(1e-8 if prec == "f64" else 3e-4) if theta is None else theta,
                        fallback=fallback)
    return lat


def _pops(E, lat):
    g = torch.empty((9, lat.dims[1], lat.dims[0]), dtype=torch.float64, device="cuda")
    E.elbm2d_read_populations(lat.h, g)
    torch.cuda.synchronize()
    return g.cpu()


@pytest.mark.parametrize("dims", [(300, 7), (33, 40), (8, 3), (256, 5)])
@pytest.mark.parametrize("kind", ["uniform", "fields"])
def test_fp64_node_by_node(E, dims, kind):
    nx, ny = dims
    uf, D3, phi0 = _fields(nx, ny, nx + ny)
    if kind == "uniform":
        u = (0.05, -0.03)
        D = _rot2(0.7) @ np.diag([0.05, 2e-4]) @ _rot2(0.7).T
        lat = _lattice(E, dims, "f64", u=u, D=D)
        prob = O2.Problem.from_tensor(u, D, theta=1e-8)
        u0 = u
    else:
        lat = _lattice(E, dims, "f64", ufield=uf, D3=D3)
        uf32 = torch.as_tensor(uf.astype(np.float32).astype(np.float64))
        prob = O2.Problem(u=uf32, S=_S_field(D3.astype(np.float32).astype(np.float64)), theta=1e-8)
        u0 = uf32
    E.elbm2d_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    ref = O2.init_equilibrium(phi0, u0)
    for n in range(12):
        E.elbm2d_step(lat.h, 1)
        ref = O2.step(ref, prob)
        if n in (0, 3, 11):
            g = _pops(E, lat)
            err = (g - ref).abs().max().item() / ref.abs().max().item()
            assert err < 1e-12, (n, err)
    d = E.elbm2d_reduce(lat.h)
    od = O2.diagnostics(ref)
    assert d["mass"] == pytest.approx(od["mass"], rel=1e-13)
    assert d["entropy"] == pytest.approx(od["entropy"], rel=1e-12)
    assert d["gmin"] == pytest.approx(od["gmin"], rel=1e-12)
    assert d["n_fallback"] == prob.stats["fallback_nodes"]
    lat.close()


def test_fp64_fallback_counts(E):
    """Adversarial step function, weak axis 1e-6, u = (0.1, 0.05): the fallback fires; the GPU
    takes it at the same node collisions as the oracle and the populations stay >= 0 up to the
    rounding of g + alpha Omega (1e-15 of the largest population)."""
    nx, ny = 40, 12
    x = np.ones((ny, 1)) * np.arange(nx)[None, :]
    phi0 = np.where(x < 20, 1.0, 1e-6)
    u, D = (0.1, 0.05), _rot2(0.5) @ np.diag([0.05, 1e-6]) @ _rot2(0.5).T
    lat = _lattice(E, (nx, ny), "f64", u=u, D=D)
    E.elbm2d_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    prob = O2.Problem.from_tensor(u, D, theta=1e-8)
    ref = O2.run(O2.init_equilibrium(phi0, u), prob, 25)
    E.elbm2d_step(lat.h, 25)
    g = _pops(E, lat)
    d = E.elbm2d_reduce(lat.h)
    assert prob.stats["fallback_nodes"] > 0
    assert d["n_fallback"] == prob.stats["fallback_nodes"]
    assert d["gmin"] >= -1e-15 * ref.abs().max().item()
    assert (g - ref).abs().max().item() / ref.abs().max().item() < 1e-12
    lat.close()


@pytest.mark.parametrize("dims", [(300, 7), (64, 48)])
def test_fp32_against_fp64_oracle(E, dims):
    nx, ny = dims
    uf, D3, phi0 = _fields(nx, ny, 3)
    lat = _lattice(E, dims, "f32", ufield=uf, D3=D3)
    E.elbm2d_init_equilibrium(lat.h, torch.as_tensor(phi0, dtype=torch.float32, device="cuda"))
    E.elbm2d_step(lat.h, 30)
    phi = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    E.elbm2d_read_moments(lat.h, phi)
    torch.cuda.synchronize()
    uf32 = torch.as_tensor(uf.astype(np.float32).astype(np.float64))
    prob = O2.Problem(u=uf32, S=_S_field(D3.astype(np.float32).astype(np.float64)), theta=3e-4)
    ref = O2.run(O2.init_equilibrium(phi0.astype(np.float32).astype(np.float64), uf32), prob, 30).sum(0)
    err = float(torch.linalg.vector_norm(phi.cpu() - ref) / torch.linalg.vector_norm(ref))
    assert err < 2e-6, err
    lat.close()


def test_fp32_large_velocity_tables(E):
    """Per-node velocities up to |u| = 0.2: the FP32 tables of a node's own u switch from the
    artanh series to logf where |s| = |t / (2 + t)| > 0.3 (|c.u| about 0.24 and above), so both
    branches are taken in one lattice; phi after 20 steps against the FP64 oracle with the same
    fields, to the FP32 bound of the other D2Q9 tests."""
    nx, ny = 64, 48
    uf, D3, phi0 = _fields(nx, ny, 5)
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    amp = 0.1 + 0.1 * np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * y / ny)      # 0 .. 0.2
    uf = np.stack([amp * np.cos(0.6), amp * np.sin(0.6)])
    cu = np.abs(uf[0]) + np.abs(uf[1])
    t = 3 * cu + 4.5 * cu ** 2 - 1.5 * (uf ** 2).sum(0)
    assert (np.abs(t / (2 + t)) > 0.3).mean() > 0.05 and (np.abs(t / (2 + t)) <= 0.3).mean() > 0.5
    lat = _lattice(E, (nx, ny), "f32", ufield=uf, D3=D3)
    E.elbm2d_init_equilibrium(lat.h, torch.as_tensor(phi0, dtype=torch.float32, device="cuda"))
    E.elbm2d_step(lat.h, 20)
    phi = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    E.elbm2d_read_moments(lat.h, phi)
    torch.cuda.synchronize()
    uf32 = torch.as_tensor(uf.astype(np.float32).astype(np.float64))
    prob = O2.Problem(u=uf32, S=_S_field(D3.astype(np.float32).astype(np.float64)), theta=3e-4)
    ref = O2.run(O2.init_equilibrium(phi0.astype(np.float32).astype(np.float64), uf32), prob, 20).sum(0)
    err = float(torch.linalg.vector_norm(phi.cpu() - ref) / torch.linalg.vector_norm(ref))
    assert err < 2e-6, err
    lat.close()


def test_arguments(E):
    L = E.lib()
    import ctypes as C
    h = C.c_void_p()
    assert L.elbm2d_create((C.c_int64 * 2)(65536, 32768), 1, None, C.byref(h)) == 1      # N >= 2^31
    assert L.elbm2d_create((C.c_int64 * 2)(16, 16), 2, None, C.byref(h)) == 9            # deviation storage
    assert L.elbm2d_create((C.c_int64 * 2)(0, 16), 1, None, C.byref(h)) == 1
    lat = E.Lattice2D((16, 8), "f32")
    with pytest.raises(E.ElbmError) as ei:
        E.elbm2d_set_tensor_uniform(lat.h, [1e-2, 2e-2, 1e-2])                          # not SPD
    assert ei.value.status == 2
    with pytest.raises(E.ElbmError) as ei:
        E.elbm2d_set_velocity_uniform(lat.h, [0.9, 0.0])                                # P_i <= 0
    assert ei.value.status == 3
    with pytest.raises(E.ElbmError) as ei:
        E.elbm2d_step(lat.h, 1)                                                          # not initialised
    assert ei.value.status == 8
    bad = np.ones((3, 8, 16), dtype=np.float32) * 1e-2
    bad[1, 3, 4] = 5e-2                                                                  # one non-SPD node
    with pytest.raises(E.ElbmError) as ei:
        E.elbm2d_set_tensor_field(lat.h, bad)
    assert ei.value.status == 2
    E.elbm2d_set_tensor_uniform(lat.h, [1e-2, 0.0, 1e-3])
    g = np.random.default_rng(0).uniform(0.01, 0.1, (9, 8, 16))
    E.elbm2d_write_populations(lat.h, g)
    back = np.empty_like(g)
    E.elbm2d_read_populations(lat.h, back)
    assert np.array_equal(back, g.astype(np.float32).astype(np.float64))
    lat.close()


def test_fullsize_sampled_one_step(E):
    """4096 x 4096 FP32 (the size bench.py times), per-node fields: one step on the GPU, and
    for 4000 random nodes plus every node of the rows y = 0, y = Ny - 1 and columns x = 0,
    x = Nx - 1 (the periodic wraps) the oracle collides the 3 x 3 source patch of the GPU's
    own pre-step populations in FP64 and streams it to the node.  Bound: FP32 rounding of one
    step, 2e-6 of the node's largest population."""
    nx = ny = 4096
    uf, D3, phi0 = _fields(nx, ny, 11)
    lat = _lattice(E, (nx, ny), "f32", ufield=uf, D3=D3)
    E.elbm2d_init_equilibrium(lat.h, torch.as_tensor(phi0, dtype=torch.float32, device="cuda"))
    E.elbm2d_step(lat.h, 5)
    before = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    E.elbm2d_read_populations(lat.h, before)
    E.elbm2d_step(lat.h, 1)
    after = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    E.elbm2d_read_populations(lat.h, after)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.integers(0, nx, 4000), np.arange(nx), np.arange(nx), np.zeros(ny, int), np.full(ny, nx - 1)])
    ys = np.concatenate([rng.integers(0, ny, 4000), np.zeros(nx, int), np.full(nx, ny - 1), np.arange(ny), np.arange(ny)])
    uf32 = uf.astype(np.float32).astype(np.float64)
    D332 = D3.astype(np.float32).astype(np.float64)
    worst = 0.0
    for c0 in range(0, len(xs), 4096):
        X, Y = xs[c0:c0 + 4096], ys[c0:c0 + 4096]
        # source nodes of every population: (x - cx, y - cy)
        pre, uu, DD = [], [], []
        for i, (cx, cy) in enumerate(O2.C_INT):
            sx, sy = (X - cx) % nx, (Y - cy) % ny
            idx = torch.as_tensor(sy * nx + sx, device="cuda")
            pre.append(before.reshape(9, -1)[:, idx].cpu())
            uu.append(uf32.reshape(2, -1)[:, sy * nx + sx])
            DD.append(D332.reshape(3, -1)[:, sy * nx + sx])
        g = torch.stack(pre, 1)                                  # [9 pops, 9 sources, M]
        uv = torch.as_tensor(np.stack(uu, 1))                    # [2, 9, M]
        S = _S_field(np.stack(DD, 1))                            # [9, M, 2, 2]
        post, _ = O2.collide(g, uv, S, theta=3e-4, lam_mode="reduced")
        ref = torch.stack([post[i, i] for i in range(9)])       # population i from source i
        got = after.reshape(9, -1)[:, torch.as_tensor(Y * nx + X, device="cuda")].cpu()
        err = ((got - ref).abs().max(0).values / ref.abs().max(0).values).max().item()
        worst = max(worst, err)
    assert worst < 2e-6, worst
    lat.close()
