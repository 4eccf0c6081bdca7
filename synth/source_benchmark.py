"""Inputs of the source-driven variable-tensor benchmark of Section 3.3 (input recipe only).

Physical box [0,1)^3 on n^3 nodes x_i = i/n, dx = 1/n, dt = dx^2 (so lattice and physical
diffusivities coincide), u = (1,1,1) -> lattice velocity dx * u.  K = diag(d1 (2 - S), d2, d3)
with S = sin(2 pi x) sin(2 pi y) sin(2 pi z); exact solution phi = exp(A t) S with
A = 1 - 4 pi^2 (2 d1 + d2 + d3); source R = exp(A t) f(x) with
f = S + 4 d1 pi^2 cos(4 pi x) sin^2(2 pi y) sin^2(2 pi z) + 2 pi (u . grad-part).
The computation carries the shifted scalar psi = phi + shift.
"""
import math

import numpy as np


def setup(n=128, d=(1e-2, 1e-2, 1e-6), u=(1.0, 1.0, 1.0), shift=2.0, t_end=3.0):
    dx = 1.0 / n
    dt = dx * dx
    ax = np.arange(n) * dx
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    sx, sy, sz = np.sin(2 * math.pi * x), np.sin(2 * math.pi * y), np.sin(2 * math.pi * z)
    cx, cy, cz = np.cos(2 * math.pi * x), np.cos(2 * math.pi * y), np.cos(2 * math.pi * z)
    S = sx * sy * sz
    d1, d2, d3 = d
    A = 1.0 - 4.0 * math.pi ** 2 * (2 * d1 + d2 + d3)
    f = (S + 4.0 * d1 * math.pi ** 2 * np.cos(4 * math.pi * x) * sy ** 2 * sz ** 2
         + 2.0 * math.pi * (u[0] * cx * sy * sz + u[1] * sx * cy * sz + u[2] * sx * sy * cz))
    D6 = np.zeros((6, n, n, n))
    D6[0] = d1 * (2.0 - S)
    D6[3] = d2
    D6[5] = d3
    steps = int(round(t_end / dt))
    amp = dt * np.exp(A * (np.arange(steps) + 0.5) * dt)      # R at t_{n+1/2}, times dt
    return dict(n=n, dims=(n, n, n), dt=dt, A=A, S=S, f=f, D6=D6, psi0=shift + S, shift=shift,
                u_lat=np.asarray(u) * dx, steps=steps, amp=amp,
                exact=lambda t: math.exp(A * t) * S)
