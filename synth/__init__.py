"""Seeded synthetic inputs for the anisotropic ADE lattice Boltzmann workloads.

This module only *produces inputs*: initial scalar fields, diffusion tensors
built from principal values and Euler angles, porous masks, rotation fields,
source fields and batched-domain tables.  It holds none of the lattice
Boltzmann arithmetic (no velocity set, no equilibrium, no collision, no
streaming).  Both the CUDA path and the FP64 oracle consume what it returns;
neither side imports the other.

All randomness comes from ``numpy.random.Generator(PCG64(seed))`` so a seed
fixes every array.  Arrays are ``float64`` numpy arrays laid out
``[..., Nz, Ny, Nx]`` (x fastest), the layout the library uses on the device.

Tensor convention (Section 3.1, Gaussian benchmark): ZYZ Euler angles,
``R = Rz(a) Ry(b) Rz(g)`` with active right-handed rotations, and
``D = R diag(d1, d2, d3) R^T``.  The Cartesian 6-vector order is
``(Dxx, Dxy, Dxz, Dyy, Dyz, Dzz)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

D6_ORDER = ("xx", "xy", "xz", "yy", "yz", "zz")


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# Rotations and tensors (input recipe of Sections 3.1, 3.2 and 4.2.1)
# ----------------------------------------------------------------------------
def rot_z(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_y(b: float) -> np.ndarray:
    c, s = math.cos(b), math.sin(b)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def rot_zyz(a: float, b: float, g: float) -> np.ndarray:
    """ZYZ rotation R = Rz(a) Ry(b) Rz(g) (angles in radians)."""
    return rot_z(a) @ rot_y(b) @ rot_z(g)


def rot_zyz_deg(a: float, b: float, g: float) -> np.ndarray:
    return rot_zyz(math.radians(a), math.radians(b), math.radians(g))


def tensor_from_principal(d, R: np.ndarray) -> np.ndarray:
    """D = R diag(d) R^T for principal values d (3,) and rotation R (3, 3)."""
    return R @ np.diag(np.asarray(d, dtype=np.float64)) @ R.T


def haar_euler(g: np.random.Generator):
    """Uniformly random orientation as ZYZ angles: a, c ~ U[0, 2pi), b = arccos U[-1, 1]."""
    a = g.uniform(0.0, 2.0 * math.pi)
    b = math.acos(g.uniform(-1.0, 1.0))
    c = g.uniform(0.0, 2.0 * math.pi)
    return a, b, c


def d6_from_matrix(D: np.ndarray) -> np.ndarray:
    """(..., 3, 3) symmetric -> (..., 6) in (xx, xy, xz, yy, yz, zz) order."""
    return np.stack([D[..., 0, 0], D[..., 0, 1], D[..., 0, 2],
                     D[..., 1, 1], D[..., 1, 2], D[..., 2, 2]], axis=-1)


def matrix_from_d6(d6: np.ndarray) -> np.ndarray:
    d6 = np.asarray(d6, dtype=np.float64)
    xx, xy, xz, yy, yz, zz = (d6[..., k] for k in range(6))
    return np.stack([np.stack([xx, xy, xz], -1),
                     np.stack([xy, yy, yz], -1),
                     np.stack([xz, yz, zz], -1)], -2)


# ----------------------------------------------------------------------------
# Scalar fields
# ----------------------------------------------------------------------------
def grid(dims):
    """Node coordinates (x, y, z) as [Nz, Ny, Nx] arrays; dims = (Nx, Ny, Nz)."""
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def sine_mode(dims, m, c0=1.0, amp=0.1, fn=np.sin):
    """c0 + amp * fn(k . x), k = 2 pi (mx/Nx, my/Ny, mz/Nz)."""
    x, y, z = grid(dims)
    k = [2.0 * math.pi * m[a] / dims[a] for a in range(3)]
    return c0 + amp * fn(k[0] * x + k[1] * y + k[2] * z)


def gaussian(dims, mu, sigma, peak=1.0):
    """Isotropic Gaussian of width sigma centred at mu (no periodic images)."""
    x, y, z = grid(dims)
    r2 = (x - mu[0]) ** 2 + (y - mu[1]) ** 2 + (z - mu[2]) ** 2
    return peak * np.exp(-0.5 * r2 / sigma ** 2)


def smooth_noise(dims, g: np.random.Generator, sigma: float) -> np.ndarray:
    """White noise low-passed by a periodic Gaussian filter of width sigma nodes."""
    nx, ny, nz = dims
    sigma = min(sigma, min(dims) / 6.0)      # keep some variance on small boxes
    w = g.standard_normal((nz, ny, nx))
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.fftfreq(nx)[None, None, :]
    filt = np.exp(-2.0 * (math.pi * sigma) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    out = np.real(np.fft.ifftn(np.fft.fftn(w) * filt))
    out -= out.mean()
    return out / max(out.std(), 1e-12)


def porous_mask(dims, seed: int, porosity=0.6, sigma=3.0) -> np.ndarray:
    """Two-phase mask (True = pore): filtered noise thresholded at its porosity quantile."""
    f = smooth_noise(dims, rng(seed), sigma)
    thr = np.quantile(f, porosity)
    return f <= thr


# ----------------------------------------------------------------------------
# Workload configurations (sizes and recipes, see the design notes)
# ----------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    dims: tuple
    steps: int
    u: np.ndarray                    # (3,) uniform velocity
    D: np.ndarray | None = None      # (3, 3) uniform tensor, or None
    D6_field: np.ndarray | None = None  # (6, Nz, Ny, Nx) per-node tensor
    phi0: np.ndarray | None = None   # (Nz, Ny, Nx)
    source: np.ndarray | None = None  # (Nz, Ny, Nx) time-constant volumetric rate R
    dirichlet_x: tuple | None = None  # (phi at x = -1/2, phi at x = Nx - 1/2)
    meta: dict = field(default_factory=dict)


def decay_mode(n=32, seed=1, eig=(0.05, 0.005, 0.0005), steps=200, m=(1, 1, 0),
               euler=None, dims=None) -> Workload:
    """Rotated single Fourier mode, u = 0 (Section 3.2 shape).

    phi0 = 1 + 0.1 sin(k.x), D = R diag(eig) R^T with Haar-random R from `seed`
    (or fixed ZYZ angles in degrees via `euler`).
    """
    dims = tuple(dims) if dims is not None else (n, n, n)
    if euler is None:
        ang = haar_euler(rng(seed))
        R = rot_zyz(*ang)
    else:
        ang = tuple(math.radians(e) for e in euler)
        R = rot_zyz(*ang)
    D = tensor_from_principal(eig, R)
    return Workload(name=f"decay_mode_{dims[0]}x{dims[1]}x{dims[2]}", dims=dims, steps=steps,
                    u=np.zeros(3), D=D, phi0=sine_mode(dims, m),
                    meta=dict(eig=tuple(eig), euler=ang, m=tuple(m), seed=seed))


def gaussian_plume(n=256, seed=2, eig=(0.1, 1e-3, 1e-5), u=(0.05, 0.03, 0.02), sigma0=8.0,
                   steps=2000, dims=None) -> Workload:
    """Advected anisotropic Gaussian plume (Section 3.1 shape), periodic box."""
    dims = tuple(dims) if dims is not None else (n, n, n)
    ang = haar_euler(rng(seed))
    D = tensor_from_principal(eig, rot_zyz(*ang))
    mu0 = tuple((d - 1) / 2.0 for d in dims)
    return Workload(name=f"gaussian_plume_{dims[0]}x{dims[1]}x{dims[2]}", dims=dims, steps=steps,
                    u=np.asarray(u, dtype=np.float64), D=D, phi0=gaussian(dims, mu0, sigma0),
                    meta=dict(eig=tuple(eig), euler=ang, sigma0=sigma0, mu0=mu0, seed=seed))


PORE_EIG = (3e-2, 3e-3, 1e-6)
SOLID_EIG = (1e-2, 1e-4, 1e-6)


def heterogeneous(n=384, seed=3, steps=50, porosity=0.6, src_amp=1e-4, src_width=16.0,
                  dims=None, shift=1.0) -> Workload:
    """Two-phase porous medium with a smooth rotation field, Gaussian source and
    Dirichlet x-faces (phi = 1 + shift at x = -1/2, phi = shift at x = Nx - 1/2); u = 0.

    The scalar is shifted by a constant, as Section 3.3 does for fields that would reach
    zero, so that the populations stay positive: with shift = 0 the outlet face keeps the
    positivity fallback firing and the run does not reach steady state.

    Pore principal values (3e-2, 3e-3, 1e-6), solid (1e-2, 1e-4, 1e-6): the
    largest local contrast is 3e-2 / 1e-6 = 3e4.  The ZYZ angles vary as
    e0 + 0.5 sin(2 pi k_r . x / N + p_r) per angle with seeded e0, k_r, p_r.
    """
    dims = tuple(dims) if dims is not None else (n, n, n)
    g = rng(seed)
    mask = porous_mask(dims, seed, porosity=porosity, sigma=3.0)
    x, y, z = grid(dims)
    ang = []
    for _ in range(3):
        e0 = g.uniform(0.0, 2.0 * math.pi)
        kr = g.integers(1, 3, size=3)
        pr = g.uniform(0.0, 2.0 * math.pi)
        ang.append(e0 + 0.5 * np.sin(2 * math.pi * (kr[0] * x / dims[0] + kr[1] * y / dims[1]
                                                       + kr[2] * z / dims[2]) + pr))
    a, b, c = ang
    ca, sa, cb, sb, cc, sc = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)
    del ang, a, b, c
    # R = Rz(a) Ry(b) Rz(c), written out per node as its nine entries R[r][k]
    R = [[ca * cb * cc - sa * sc, -ca * cb * sc - sa * cc, ca * sb],
         [sa * cb * cc + ca * sc, -sa * cb * sc + ca * cc, sa * sb],
         [-sb * cc, sb * sc, cb]]
    lam = [np.where(mask, PORE_EIG[k], SOLID_EIG[k]) for k in range(3)]
    # D = R diag(lam) R^T, the six components (xx, xy, xz, yy, yz, zz)
    D6 = np.empty((6,) + dims[::-1])
    for q, (r1, r2) in enumerate(((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
        D6[q] = R[r1][0] * lam[0] * R[r2][0] + R[r1][1] * lam[1] * R[r2][1] + R[r1][2] * lam[2] * R[r2][2]
    del R, lam
    mu = tuple((d - 1) / 2.0 for d in dims)
    src = gaussian(dims, mu, src_width, peak=src_amp)
    # linear initial profile between the two Dirichlet values
    phi0 = shift + 1.0 - (x + 0.5) / dims[0]
    return Workload(name=f"heterogeneous_{dims[0]}x{dims[1]}x{dims[2]}", dims=dims, steps=steps,
                    u=np.zeros(3), D6_field=D6, phi0=phi0, source=src, dirichlet_x=(1.0 + shift, shift),
                    meta=dict(mask=mask, seed=seed, porosity=float(mask.mean()), shift=shift))


def batched_domains(ndom=512, seed=4, nmin=16, nmax=96, steps=500):
    """Table of independent periodic domains for the orientation/anisotropy sweep.

    Each entry: edge n ~ U{nmin..nmax}; Haar-random orientation; anisotropy
    r log-uniform in [1, 1e4]; principal values (0.05, 0.05/sqrt(r), 0.05/r);
    initial field 1 + 0.1 sin(k.x) with k = 2 pi (1, 1, 0) / n; u = 0.
    """
    g = rng(seed)
    out = []
    for d in range(ndom):
        n = int(g.integers(nmin, nmax + 1))
        ang = haar_euler(g)
        r = 10.0 ** g.uniform(0.0, 4.0)
        eig = (0.05, 0.05 / math.sqrt(r), 0.05 / r)
        D = tensor_from_principal(eig, rot_zyz(*ang))
        out.append(dict(n=n, euler=ang, ratio=r, eig=eig, D=D))
    return out, steps


def batched_phi0(n):
    return sine_mode((n, n, n), (1, 1, 0))


def adjoint_problem(n=64, seed=5, steps=500, obs=(250, 500), u=(0.02, 0.0, 0.0), sigma=6.0,
                    base_eig=(1e-2, 1e-3, 1e-4), perturb=0.1):
    """Per-node tensor parameters theta = (log d1, log d2, log d3, a, b, c) on an n^3 box.

    theta* is smooth around log(base_eig) with a smooth orientation field;
    theta0 = theta* + perturb * smooth noise.  Returns (theta_true, theta0,
    phi0, u, obs) as float64 arrays [6, n, n, n] / [n, n, n].
    """
    dims = (n, n, n)
    g = rng(seed)
    th = np.empty((6,) + dims)
    for k in range(3):
        th[k] = math.log(base_eig[k]) + 0.3 * smooth_noise(dims, g, 6.0)
    for k in range(3):
        th[3 + k] = g.uniform(0.0, 2.0 * math.pi) + 0.5 * smooth_noise(dims, g, 6.0)
    th0 = th + perturb * np.stack([smooth_noise(dims, g, 4.0) for _ in range(6)])
    mu = tuple((d - 1) / 2.0 for d in dims)
    phi0 = 0.1 + gaussian(dims, mu, sigma)
    return dict(theta_true=th, theta0=th0, phi0=phi0, u=np.asarray(u, np.float64),
                obs=tuple(obs), steps=steps, dims=dims)


def channel2d(nx=4096, ny=4096, seed=11, U=0.04, drift=0.01, d1=0.03, steps=200):
    """Two-dimensional fields shaped like Section 4.1's channel problem on a periodic box:
    a streamwise velocity U (1 + sin(2 pi (y + 1/2)/Ny))/2 with a weaker wall-normal drift
    -drift cos(2 pi y / Ny), and a tensor whose principal values and orientation vary across
    the channel (d1 (1 + 0.3 s), d2 (1 + 0.2 cos), angle 0.6 + 0.8 s + 0.1 sin(2 pi x / Nx),
    s = sin(2 pi (y + 1/2)/Ny), d2 log-uniform in [1e-4, 1e-2] from `seed`); initial field
    1 + a Gaussian bump.  Returns (u [2, Ny, Nx], D3 [3, Ny, Nx] as (Dxx, Dxy, Dyy), phi0)."""
    g = rng(seed)
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    x = np.ones((ny, 1)) * np.arange(nx, dtype=np.float64)[None, :]
    s = np.sin(2 * math.pi * (y + 0.5) / ny)
    u = np.stack([U * (0.5 + 0.5 * s), -drift * np.cos(2 * math.pi * y / ny)])
    ang = 0.6 + 0.8 * s + 0.1 * np.sin(2 * math.pi * x / nx)
    a = d1 * (1 + 0.3 * s)
    b = 10 ** g.uniform(-4, -2) * (1 + 0.2 * np.cos(2 * math.pi * y / ny))
    c, sn = np.cos(ang), np.sin(ang)
    D3 = np.stack([c * c * a + sn * sn * b, c * sn * (a - b), sn * sn * a + c * c * b])
    phi0 = 1.0 + 0.5 * np.exp(-((x - nx / 2) ** 2 / (2 * (nx / 6) ** 2) + (y - ny / 2) ** 2 / (2 * (ny / 5) ** 2)))
    return u, D3, phi0
