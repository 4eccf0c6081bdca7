"""Pin of the advective part of the oracle against the analytic anisotropic
Gaussian (Section 3.1): centroid mu0 + u t and covariance Sigma0 + 2 D t (P5),
plus exact mass conservation (P6).

The equilibrium start excites a short flux transient that shifts the
covariance by a constant, so D is recovered from the covariance difference
between two times, t1 = 40 and t2 = 80."""
import numpy as np
import pytest

import oracle as O
import synth


def plume_moments(phi, center):
    nz, ny, nx = phi.shape
    x, y, z = synth.grid((nx, ny, nz))
    X, N = [x, y, z], [nx, ny, nz]
    d = [((X[a] - center[a] + N[a] / 2) % N[a]) - N[a] / 2 for a in range(3)]
    M = phi.sum()
    mu = np.array([(phi * d[a]).sum() / M for a in range(3)])
    cov = np.array([[(phi * (d[a] - mu[a]) * (d[b] - mu[b])).sum() / M for b in range(3)]
                    for a in range(3)])
    return M, mu + np.asarray(center), cov


def test_gaussian_plume_moments():
    wl = synth.gaussian_plume(n=40, sigma0=5.0, eig=(0.05, 0.01, 0.002), steps=80)
    prob = O.Problem.from_tensor(wl.u, wl.D)
    g = O.init_equilibrium(wl.phi0, wl.u)
    snaps = {}
    O.run(g, prob, 80, callback=lambda k, g: snaps.__setitem__(k, g.sum(0).numpy()) if k in (40, 80) else None)
    mu0 = np.asarray(wl.meta["mu0"])
    m1 = plume_moments(snaps[40], mu0 + wl.u * 40)
    m2 = plume_moments(snaps[80], mu0 + wl.u * 80)
    M0 = wl.phi0.sum()
    assert abs(m2[0] - M0) / M0 < 1e-13                       # mass (P6)
    u_rec = (m2[1] - m1[1]) / 40.0
    assert np.abs(u_rec - wl.u).max() < 1e-4                  # centroid speed = u
    assert np.abs(m2[1] - (mu0 + 80 * wl.u)).max() < 2e-3      # centroid position
    D_rec = (m2[2] - m1[2]) / (2 * 40.0)
    err = np.abs(D_rec - wl.D).max() / np.abs(wl.D).max()
    assert err < 1e-2, err                                   # measured 7.2e-3 at this resolution
