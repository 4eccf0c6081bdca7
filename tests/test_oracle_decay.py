"""Pins of the full oracle step at zero velocity against the exact Fourier
recurrence (P2) and the continuum decay law exp(-k.Dk t) (P3)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from fourier_pin import dominant_rate, mode_history


def _run_modes(wl, nsteps, m):
    prob = O.Problem.from_tensor(wl.u, wl.D)
    g = O.init_equilibrium(wl.phi0, wl.u)
    idx = (m[2] % wl.dims[2], m[1] % wl.dims[1], m[0] % wl.dims[0])
    hist = []
    O.run(g, prob, nsteps, callback=lambda n, g: hist.append(np.fft.fftn(g.sum(0).numpy())[idx]))
    return np.array(hist), prob


@pytest.mark.parametrize("dims,m,seed", [((12, 10, 8), (1, 2, 1), 1), ((16, 16, 16), (1, 1, 0), 1),
                                         ((9, 7, 5), (2, -1, 1), 7)])
def test_exact_fourier_recurrence(dims, m, seed):
    """Non-cubic grids and oblique modes catch swapped axes and streaming signs."""
    wl = synth.decay_mode(dims=dims, seed=seed, m=m, steps=60)
    hist, prob = _run_modes(wl, 60, m)
    k = 2 * math.pi * np.asarray(m, float) / np.asarray(dims, float)
    S = np.linalg.inv(0.5 * np.eye(3) + 3.0 * wl.D)
    idx = (m[2] % dims[2], m[1] % dims[1], m[0] % dims[0])
    pred = mode_history(k, S, np.fft.fftn(wl.phi0)[idx], 60)
    scale = abs(np.fft.fftn(wl.phi0)[idx])
    assert np.max(np.abs(hist - pred)) / scale < 1e-12
    assert prob.stats["fallback_nodes"] == 0


def test_config1_decay_32cubed():
    """32^3, u = 0, seeded rotation, 200 steps: exact recurrence to 1e-12 and
    the fitted rate within 1e-2 of k.Dk (discretisation error ~4e-3 at k = 2pi/32)."""
    wl = synth.decay_mode(n=32, seed=1, steps=200)
    m = (1, 1, 0)
    hist, prob = _run_modes(wl, 200, m)
    k = 2 * math.pi * np.asarray(m, float) / 32
    S = np.linalg.inv(0.5 * np.eye(3) + 3.0 * wl.D)
    pred = mode_history(k, S, np.fft.fftn(wl.phi0)[0, 1, 1], 200)
    scale = abs(np.fft.fftn(wl.phi0)[0, 1, 1])
    assert np.max(np.abs(hist - pred)) / scale < 1e-12
    t = np.arange(1, 201)
    sl = slice(100, 200)        # after the fast flux transients of the equilibrium start
    rate = -np.polyfit(t[sl], np.log(np.abs(hist[sl])), 1)[0]
    theory = k @ wl.D @ k
    assert abs(rate - theory) / theory < 1e-2
    assert abs(rate - dominant_rate(k, S)) / theory < 1e-4     # residual fast-mode transients
    mass0 = wl.phi0.sum()
    assert abs(hist.shape[0] - 200) == 0
    assert abs(O.diagnostics(O.init_equilibrium(wl.phi0, wl.u))["mass"] - mass0) < 1e-12 * mass0


def test_table2_mode_on_paper_grid():
    """Paper's decay grid 256 x 256 (z-independent mode, so Nz = 1 is exact),
    case 10^4:10^2:1 at (120, 90, 135): the oracle follows the recurrence whose
    rate is Table 2's alpha_ELBM."""
    dims = (256, 256, 1)
    wl = synth.decay_mode(dims=dims, eig=(1e-2, 1e-4, 1e-6), euler=(120, 90, 135), m=(3, 3, 0))
    wl.phi0 = synth.sine_mode(dims, (3, 3, 0), c0=1.0, amp=1e-2, fn=np.cos)
    hist, _ = _run_modes(wl, 40, (3, 3, 0))
    k = 2 * math.pi * np.array([3, 3, 0]) / 256
    S = np.linalg.inv(0.5 * np.eye(3) + 3.0 * wl.D)
    pred = mode_history(k, S, np.fft.fftn(wl.phi0)[0, 3, 3], 40)
    assert np.max(np.abs(hist - pred)) / abs(pred[0]) < 1e-12
    assert dominant_rate(k, S) == pytest.approx(5.11329e-5, rel=1.5e-4)
