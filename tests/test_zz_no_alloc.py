"""Allocation-free diagnostics.

elbm_reduce_noalloc serves callers that cannot allocate device memory when they
want the conservation diagnostics (device memory fully reserved by another
allocator, or a monitoring hook that must not block or fail on an allocation).
Its partial sums live in a fixed device array instead of a cudaMalloc'd buffer.
It must give the same mass, entropy and minimum population as elbm_reduce, on
two calls in a row (the second call reuses the array the first one left
behind), with host and device outputs."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import gpu_lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2605_01774_gb300 import elbm
    elbm.lib()
    return elbm


@pytest.mark.parametrize("prec", ["f64", "f32", "f16dev"])
def test_noalloc_matches_reduce(E, prec):
    wl = synth.gaussian_plume(dims=(40, 24, 18), sigma0=4.0, eig=(0.05, 0.01, 0.002))
    phi0 = 0.1 + wl.phi0
    src = 1e-4 * synth.gaussian(wl.dims, (20.0, 12.0, 9.0), 3.0)
    bc = (1.2, 0.9)
    lat = gpu_lattice(E, wl.dims, prec, D=wl.D, u=wl.u, bc=bc, source=src)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(phi0, device="cuda"))
    src_dev = torch.as_tensor(src, dtype=torch.float32, device="cuda")   # the caller's own copy
    for call in range(2):
        E.elbm_step(lat.h, 3 + call)
        ref = E.elbm_reduce(lat.h)
        pops, scale = E.elbm_state_pointers(lat.h)
        out = E.elbm_reduce_noalloc(pops, scale, wl.dims, prec, wl.u, bc=bc, source=src_dev)
        dev_out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        E.elbm_reduce_noalloc(pops, scale, wl.dims, prec, wl.u, bc=bc, source=src_dev, out=dev_out)
        torch.cuda.synchronize()
        for o in (out, dev_out.cpu().numpy()):
            assert o[0] == pytest.approx(ref["mass"], rel=1e-12)
            assert o[1] == pytest.approx(ref["entropy"], rel=1e-12)
            assert o[2] == pytest.approx(ref["gmin"], rel=1e-12, abs=1e-300)
            assert o[3] == 0.0
    lat.close()


def test_noalloc_rejects_lattices_beyond_the_limit(E):
    L = E.lib()
    out = np.zeros(4)
    u = (C.c_double * 3)(0.0, 0.0, 0.0)
    dummy = torch.zeros(16, device="cuda")
    for dims in ((65536, 1, 1), (1024, 1024, 100)):
        d = (C.c_int64 * 3)(*dims)
        s = L.elbm_reduce_noalloc(C.c_void_p(dummy.data_ptr()), None, d, 1, u, None, None, None,
                                  C.c_void_p(out.ctypes.data))
        assert s == 1          # ELBM_ERR_ARG, nothing launched


def test_noalloc_rejects_host_pointers(E):
    """pops, scale and source are read by the kernels directly: host memory (pageable or
    pinned) is refused with ELBM_ERR_ARG before anything is launched."""
    L = E.lib()
    dims = (8, 4, 3)
    N = 8 * 4 * 3
    d = (C.c_int64 * 3)(*dims)
    u = (C.c_double * 3)(0.0, 0.0, 0.0)
    out = np.zeros(4)
    host_pops = np.zeros(27 * N, dtype=np.float32)
    pinned = torch.zeros(27 * N, dtype=torch.float32).pin_memory()
    dev_pops = torch.zeros(27 * N, dtype=torch.float32, device="cuda")
    dev_scale = torch.ones(N, dtype=torch.float32, device="cuda")
    host_src = np.zeros(N, dtype=np.float32)
    cases = [
        (host_pops.ctypes.data, None, 1, None),              # pageable host populations
        (pinned.data_ptr(), None, 1, None),                  # pinned host populations
        (dev_pops.data_ptr(), host_src.ctypes.data, 2, None),  # host scale plane
        (dev_pops.data_ptr(), None, 1, host_src.ctypes.data),  # host source plane
    ]
    for pops, scale, prec, src in cases:
        s = L.elbm_reduce_noalloc(C.c_void_p(pops), C.c_void_p(scale) if scale else None, d, prec, u, None,
                                  C.c_void_p(src) if src else None, None, C.c_void_p(out.ctypes.data))
        assert s == 1
    # the same call with device memory is accepted
    s = L.elbm_reduce_noalloc(C.c_void_p(dev_pops.data_ptr()), C.c_void_p(dev_scale.data_ptr()), d, 2, u, None,
                              None, None, C.c_void_p(out.ctypes.data))
    assert s == 0


@pytest.mark.parametrize("prec", ["f64", "f16dev"])
def test_noalloc_with_source_amplitude_schedule(E, prec):
    """A time-dependent source amplitude (Section 3.3): the stored state includes the half-step
    with the amplitude of the last step, so the caller passes that amplitude times R.  The
    amplitudes are powers of two, so the caller's FP32 product a R is exact and the two calls
    differ only in summation order."""
    wl = synth.gaussian_plume(dims=(24, 16, 12), sigma0=3.0, eig=(0.05, 0.01, 0.002))
    src = 1e-3 * synth.gaussian(wl.dims, (12.0, 8.0, 6.0), 2.5)
    lat = gpu_lattice(E, wl.dims, prec, D=wl.D, u=wl.u, source=src)
    E.elbm_set_source_amplitude(lat.h, 0.5)
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(0.2 + wl.phi0, device="cuda"))
    src_dev = torch.as_tensor(src, dtype=torch.float32, device="cuda")
    for amps in ([0.5], [2.0, 4.0, 0.25]):
        if len(amps) > 1:
            E.elbm_step_source_schedule(lat.h, amps)
        ref = E.elbm_reduce(lat.h)
        pops, scale = E.elbm_state_pointers(lat.h)
        out = E.elbm_reduce_noalloc(pops, scale, wl.dims, prec, wl.u, source=src_dev * amps[-1])
        assert out[0] == pytest.approx(ref["mass"], rel=1e-12)
        assert out[1] == pytest.approx(ref["entropy"], rel=1e-12)
        assert out[2] == pytest.approx(ref["gmin"], rel=1e-12, abs=1e-300)
    lat.close()


def test_noalloc_on_velocity_field_handle(E):
    """A handle with a per-node velocity field: its deviation storage encodes against the
    zero-velocity shape, and the call is made with u = (0, 0, 0)."""
    dims = (20, 12, 10)
    x, y, z = synth.grid(dims)
    uf = np.stack([0.04 * np.sin(2 * np.pi * y / 12), 0.03 * np.cos(2 * np.pi * z / 10),
                   0.02 * np.sin(2 * np.pi * x / 20)])
    wl = synth.gaussian_plume(dims=dims, sigma0=3.0, eig=(0.05, 0.01, 0.002))
    lat = gpu_lattice(E, dims, "f16dev", D=wl.D)
    E.elbm_set_velocity_field(lat.h, torch.as_tensor(uf, dtype=torch.float32, device="cuda"))
    E.elbm_init_equilibrium(lat.h, torch.as_tensor(0.2 + wl.phi0, device="cuda"))
    E.elbm_step(lat.h, 5)
    ref = E.elbm_reduce(lat.h)
    pops, scale = E.elbm_state_pointers(lat.h)
    out = E.elbm_reduce_noalloc(pops, scale, dims, "f16dev", (0.0, 0.0, 0.0))
    assert out[0] == pytest.approx(ref["mass"], rel=1e-12)
    assert out[1] == pytest.approx(ref["entropy"], rel=1e-12)
    assert out[2] == pytest.approx(ref["gmin"], rel=1e-12, abs=1e-300)
    lat.close()
