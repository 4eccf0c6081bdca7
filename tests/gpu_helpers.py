"""Shared helpers of the GPU parity tests: run the CUDA library through the
C ABI and the oracle on the same seeded inputs."""
import numpy as np
import torch

import oracle as O
import synth

THETA = {"f64": 1e-8, "f32": 3e-4, "f16dev": 3e-4, "bf16dev": 3e-4}


def gpu_lattice(E, dims, prec, D=None, D6_field=None, u=(0, 0, 0), bc=None, source=None, theta=None,
                eps=0.0, fallback=True, params_field=None):
    lat = E.Lattice(dims, prec, bc=bc)
    if D is not None:
        E.elbm_set_tensor_uniform(lat.h, synth.d6_from_matrix(np.asarray(D)))
    if D6_field is not None:
        E.elbm_set_tensor_field(lat.h, torch.as_tensor(np.ascontiguousarray(D6_field), dtype=torch.float32,
                                                       device="cuda"))
    if params_field is not None:
        E.elbm_set_tensor_params_field(lat.h, torch.as_tensor(np.ascontiguousarray(params_field),
                                                              dtype=torch.float32, device="cuda"))
    E.elbm_set_velocity_uniform(lat.h, u)
    if source is not None:
        E.elbm_set_source(lat.h, torch.as_tensor(np.ascontiguousarray(source), dtype=torch.float32, device="cuda"))
    E.elbm_set_params(lat.h, theta=THETA[prec] if theta is None else theta, eps=eps, fallback=fallback)
    return lat


def read_pops(E, lat):
    g = torch.empty((27,) + lat.dims[::-1], dtype=torch.float64, device="cuda")
    E.elbm_read_populations(lat.h, g)
    torch.cuda.synchronize()
    return g.cpu()


def read_phi(E, lat):
    phi = torch.empty(lat.dims[::-1], dtype=torch.float64, device="cuda")
    E.elbm_read_moments(lat.h, phi)
    torch.cuda.synchronize()
    return phi.cpu()


def oracle_problem(D=None, S_field_D=None, u=(0, 0, 0), bc=None, source=None, theta=1e-8, eps=0.0, fallback=True,
                   lam_mode="reduced"):
    u = torch.as_tensor(np.asarray(u, dtype=np.float64))
    if S_field_D is not None:
        Dm = torch.as_tensor(synth.matrix_from_d6(np.moveaxis(S_field_D, 0, -1)))
        S = O.relaxation_matrix(Dm)
    else:
        S = O.relaxation_matrix(torch.as_tensor(np.asarray(D)))
    # the library takes the source as FP32: give the oracle the same rounded values
    src = None if source is None else torch.as_tensor(np.asarray(source).astype(np.float32).astype(np.float64))
    return O.Problem(u=u, S=S, dirichlet_x=bc, source=src, theta=theta, eps=eps, fallback=fallback,
                     lam_mode=lam_mode)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
