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
