"""The implementations of the fused collide-stream step (Eq. method-lbe with the collision of
Section 2): one thread per node gathering from global memory (variant 1), persistent blocks
staging the pulled x-rows in shared memory with bulk asynchronous copies and a block barrier
per row (variant 2), and persistent blocks each with a producer warp feeding a ring of row stages
through full/empty mbarriers to consumer warps that take 32-node segments (variant 3).  They
evaluate the same arithmetic in the same order, so their outputs must be bit-equal; the staged
kernels are also checked against the FP64 oracle on their own."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import gpu_lattice, oracle_problem, read_pops

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2605_01774_gb300 import elbm
    elbm.lib()
    return elbm


def _case(dims, seed):
    rng = synth.rng(seed)
    D6 = np.empty((6,) + dims[::-1])
    for idx in np.ndindex(*dims[::-1]):
        R = synth.rot_zyz(*synth.haar_euler(rng))
        D6[(slice(None),) + idx] = synth.d6_from_matrix(synth.tensor_from_principal(10 ** rng.uniform(-4, -1, 3), R))
    phi0 = 1.0 + 0.5 * synth.gaussian(dims, tuple((d - 1) / 2 for d in dims), max(1.5, min(dims) / 4))
    src = 1e-3 * rng.uniform(0, 1, dims[::-1])
    return D6, phi0, src


def _staged_variants(E, dims, prec, u=(0.0, 0.0, 0.0), ufield=False):
    """The staged-row variants (2, 3) available for this storage, row length and velocity."""
    out = []
    for v in (2, 3):
        lat = E.Lattice(dims, prec)
        if ufield:
            E.elbm_set_velocity_field(lat.h, torch.full((3,) + dims[::-1], 0.01, device="cuda"))
        else:
            E.elbm_set_velocity_uniform(lat.h, u)
        try:
            E.elbm_set_step_kernel(lat.h, v)
            out.append(v)
        except E.ElbmError as e:
            assert e.status == 9
        lat.close()
    return out


def _run(E, dims, prec, variant, steps, D6, phi0, src, bc, u, ufield=None):
    lat = gpu_lattice(E, dims, prec, D6_field=D6, u=u, bc=bc, source=src)
    if ufield is not None:
        E.elbm_set_velocity_field(lat.h, torch.as_tensor(ufield, dtype=torch.float32, device="cuda"))
    E.elbm_set_step_kernel(lat.h, variant)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    E.elbm_step(lat.h, steps)
    E.elbm_synchronize(lat.h)
    g = read_pops(E, lat)
    fb = E.elbm_reduce(lat.h)["n_fallback"]
    lat.close()
    return g, fb


@pytest.mark.parametrize("prec", ["f64", "f32", "f16dev", "bf16dev"])
@pytest.mark.parametrize("dims,bc", [((8, 3, 2), None), ((16, 6, 5), (1.2, 0.9)), ((40, 7, 3), None),
                                     ((24, 40, 30), (1.1, 1.0)), ((96, 5, 4), (1.2, 0.9)),
                                     ((136, 6, 7), None), ((104, 40, 30), (1.1, 1.0)),
                                     ((256, 4, 3), (1.2, 0.8)), ((512, 3, 2), None), ((384, 5, 3), (1.0, 0.0))])
def test_variants_bit_equal(E, prec, dims, bc):
    """Per-node tensor, u != 0, source, Dirichlet or periodic x faces.  (24, 40, 30) and
    (104, 40, 30) have more rows than resident blocks, so blocks loop over rows and reuse their
    stages; 136 nodes per row leave a partial last segment of 8 nodes in variant 3; row lengths
    256, 384 and 512 run the instantiations with the row length compiled in."""
    variants = _staged_variants(E, dims, prec, u=(0.04, -0.03, 0.02))
    if not variants:
        pytest.skip("no staged-row variant for this storage and row length")
    D6, phi0, src = _case(dims, sum(dims))
    u = (0.04, -0.03, 0.02)
    a, fa = _run(E, dims, prec, 1, 7, D6, phi0, src, bc, u)
    for v in variants:
        b, fb = _run(E, dims, prec, v, 7, D6, phi0, src, bc, u)
        assert torch.equal(a, b), (v, (a - b).abs().max().item())
        assert fa == fb, v


@pytest.mark.parametrize("prec", ["f64", "f32", "f16dev", "bf16dev"])
@pytest.mark.parametrize("dims,u", [((16, 5, 4), (0.0, 0.0, 0.0)), ((256, 3, 2), (0.03, 0.0, -0.02)),
                                    ((384, 2, 2), (0.0, 0.0, 0.0)), ((256, 9, 7), (0.0, 0.0, 0.0)),
                                    ((512, 4, 3), (0.02, 0.01, 0.0))])
def test_variants_bit_equal_uniform_velocity_no_source(E, prec, dims, u):
    """Uniform tensor (no tensor field), u = 0 and u != 0, no source."""
    rng = synth.rng(5)
    D = synth.tensor_from_principal((0.05, 0.004, 1e-4), synth.rot_zyz(*synth.haar_euler(rng)))
    phi0 = 1.0 + 0.5 * synth.gaussian(dims, tuple((d - 1) / 2 for d in dims), 2.0)
    res = []
    for v in [1] + _staged_variants(E, dims, prec, u=u):
        lat = gpu_lattice(E, dims, prec, D=D, u=u)
        E.elbm_set_step_kernel(lat.h, v)
        E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
        E.elbm_step(lat.h, 6)
        E.elbm_synchronize(lat.h)
        res.append(read_pops(E, lat))
        lat.close()
    for r in res[1:]:
        assert torch.equal(res[0], r)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16dev"])
@pytest.mark.parametrize("dims", [(16, 5, 4), (128, 5, 4)])
def test_variants_bit_equal_velocity_field(E, prec, dims):
    x, y, z = synth.grid(dims)
    uf = np.stack([0.04 * np.sin(2 * np.pi * y / dims[1]), 0.03 * np.cos(2 * np.pi * z / dims[2]),
                   0.02 * np.sin(2 * np.pi * x / dims[0])])
    D6, phi0, _ = _case(dims, 3)
    a, _ = _run(E, dims, prec, 1, 5, D6, phi0, None, None, (0, 0, 0), ufield=uf)
    for v in _staged_variants(E, dims, prec, ufield=True):
        b, _ = _run(E, dims, prec, v, 5, D6, phi0, None, None, (0, 0, 0), ufield=uf)
        assert torch.equal(a, b), v


@pytest.mark.parametrize("dims,bc,variant", [((16, 5, 3), (1.3, 0.7), 2), ((8, 4, 4), None, 2),
                                             ((104, 3, 3), (1.3, 0.7), 3), ((40, 4, 3), None, 3)])
def test_staged_rows_vs_oracle_fp64(E, dims, bc, variant):
    """Staged-row kernels against the FP64 oracle node by node (1e-13 of the maximum), 3 steps."""
    D6, phi0, src = _case(dims, 11 + dims[0])
    u = (0.03, 0.02, -0.04)
    lat = gpu_lattice(E, dims, "f64", D6_field=D6, u=u, bc=bc, source=src)
    E.elbm_set_step_kernel(lat.h, variant)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    prob = oracle_problem(S_field_D=D6.astype(np.float32).astype(np.float64), u=u, bc=bc, source=src,
                          theta=1e-8, lam_mode="literal")
    ref = O.init_equilibrium(phi0, u)
    for n in range(3):
        E.elbm_step(lat.h, 1)
        ref = O.step(ref, prob, n)
        g = read_pops(E, lat)
        diff = (g - ref).abs().max().item() / ref.abs().max().item()
        assert diff < 1e-13, (n, diff)


def test_step_kernel_arguments(E):
    lat = E.Lattice((12, 4, 4), "f32")
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_set_step_kernel(lat.h, 2)                  # nx % 8 != 0
    assert ei.value.status == 9
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_set_step_kernel(lat.h, 3)                  # nx % 8 != 0
    assert ei.value.status == 9
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_set_step_kernel(lat.h, 4)
    assert ei.value.status == 1
    E.elbm_set_step_kernel(lat.h, 1)
    E.elbm_set_step_kernel(lat.h, 0)
    big = E.Lattice((480, 2, 2), "f64")                   # two FP64 stages exceed the limit
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_set_step_kernel(big.h, 2)
    assert ei.value.status == 9
    ok = E.Lattice((472, 2, 2), "f64")
    E.elbm_set_step_kernel(ok.h, 2)


def test_automatic_choice(E):
    """The automatic choice (measured on GB300): staged rows for the FP32-arithmetic storages
    with rows of 256 nodes or more, compiled-in length or not; the per-node kernel for shorter
    rows, per-node velocity fields, the exact-root stabilizer and FP64."""
    cases = [((256, 2, 2), "f32", None, 2), ((320, 2, 2), "f16dev", None, 2), ((264, 2, 2), "bf16dev", None, 2),
             ((192, 2, 2), "f32", None, 1), ((256, 2, 2), "f64", None, 1), ((256, 2, 2), "f32", "field", 1),
             ((256, 2, 2), "f32", "root", 1)]
    for dims, prec, mode, want in cases:
        lat = E.Lattice(dims, prec)
        if mode == "field":
            E.elbm_set_velocity_field(lat.h, torch.full((3,) + dims[::-1], 0.01, device="cuda"))
        elif mode == "root":
            E.elbm_set_velocity_uniform(lat.h, (0.02, 0.01, 0.0))
            E.elbm_set_lambda_mode(lat.h, 1)
        assert E.elbm_get_step_kernel(lat.h) == want, (dims, prec, mode)
        lat.close()


@pytest.mark.parametrize("prec", ["f32", "f16dev"])
@pytest.mark.parametrize("variant", [2, 3])
def test_staging_wait_limit_timeout_and_recovery(E, prec, variant):
    """A staging wait limit far below a copy's latency makes the staged-row kernels give up:
    blocks raise their abort flag, the thread that issued the copies waits (with the full limit)
    for those still in flight, and the next synchronise reports ELBM_ERR_TIMEOUT.  Variant 2 is
    made to time out by stage barriers that expect one arrival too many (elbm_set_wait_test);
    its abort path makes that arrival before it waits for the copies.  With the limit restored the same
    handle steps normally again and matches a fresh handle bit for bit."""
    dims = (256, 16, 12)
    D6, phi0, src = _case(dims, 9)
    u = (0.04, -0.03, 0.02)
    lat = gpu_lattice(E, dims, prec, D6_field=D6, u=u, source=src)
    E.elbm_set_step_kernel(lat.h, variant)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    if variant == 2:
        # the staged-row kernel issues its first rows before any wait, so a short limit alone
        # may find them landed: its barriers are made to expect one arrival that never comes
        E.elbm_set_wait_test(lat.h, 1)
        E.elbm_set_wait_limit(lat.h, 4096)
    else:
        E.elbm_set_wait_limit(lat.h, 16)
    E.elbm_step(lat.h, 1)
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_synchronize(lat.h)
    assert ei.value.status == 7
    E.elbm_set_wait_limit(lat.h, 0)
    E.elbm_set_wait_test(lat.h, 0)
    E.elbm_synchronize(lat.h)                             # the flag was cleared
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    E.elbm_step(lat.h, 4)
    E.elbm_synchronize(lat.h)
    g = read_pops(E, lat)
    lat.close()
    ref, _ = _run(E, dims, prec, 1, 4, D6, phi0, src, None, u)
    assert torch.equal(g, ref)
