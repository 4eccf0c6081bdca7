"""Planted mistakes in the oracle (on the CPU, via monkeypatch) must be caught
by the pins: this shows the pins constrain the parts they claim to."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import oracle.elbm as E
import synth
from fourier_pin import mode_history
from test_oracle_stabilizer import _exact_root, _split, _state


def _fourier_gap():
    dims, m = (9, 7, 5), (2, -1, 1)
    wl = synth.decay_mode(dims=dims, seed=7, m=m, steps=20)
    prob = O.Problem.from_tensor(wl.u, wl.D)
    g = O.init_equilibrium(wl.phi0, wl.u)
    idx = (m[2] % dims[2], m[1] % dims[1], m[0] % dims[0])
    hist = []
    O.run(g, prob, 20, callback=lambda n, g: hist.append(np.fft.fftn(g.sum(0).numpy())[idx]))
    k = 2 * math.pi * np.asarray(m, float) / np.asarray(dims, float)
    S = np.linalg.inv(0.5 * np.eye(3) + 3.0 * wl.D)
    pred = mode_history(k, S, np.fft.fftn(wl.phi0)[idx], 20)
    return np.max(np.abs(np.array(hist) - pred)) / abs(np.fft.fftn(wl.phi0)[idx])


def _root_gap():
    u = np.array([0.05, 0.03, 0.02])
    S = np.linalg.inv(0.5 * np.eye(3) + 3 * np.diag([0.1, 1e-3, 1e-5]))
    g = _state(u, 1e-3, 0)
    _, info = O.collide(g, torch.as_tensor(u), torch.as_tensor(S), theta=0.0, fallback=False)
    geq, dh, dsp = _split(g[:, 0].numpy(), u, S)
    root = _exact_root(geq, dh, dsp)
    return abs(info.lam.item() - root) / max(1.0, abs(root))


def _centroid_speed_gap():
    """At u = 0 the scheme is parity-symmetric, so the streaming direction only
    shows through advection: the plume centroid must move by +u per step."""
    from test_oracle_gaussian import plume_moments
    wl = synth.gaussian_plume(n=16, sigma0=3.0, eig=(0.02, 0.01, 0.005), steps=10)
    prob = O.Problem.from_tensor(wl.u, wl.D)
    g = O.run(O.init_equilibrium(wl.phi0, wl.u), prob, 10)
    mu0 = np.asarray(wl.meta["mu0"])
    _, mu, _ = plume_moments(g.sum(0).numpy(), mu0)
    return np.abs((mu - mu0) / 10 - wl.u).max()


def test_unmutated_baseline():
    assert _fourier_gap() < 1e-12
    assert _root_gap() < 5e-3
    assert _centroid_speed_gap() < 1.5e-2      # start-up transient; a reversed stream gives ~2|u|


def test_reversed_streaming_is_caught(monkeypatch):
    orig = E.stream
    monkeypatch.setattr(E, "stream", lambda gp, d=None, u_wall=None: orig(gp.flip(0), d).flip(0))
    assert _centroid_speed_gap() > 5e-2


def test_missing_half_step_correction_is_caught(monkeypatch):
    monkeypatch.setattr(E, "relaxation_matrix", lambda D: torch.linalg.inv(D / E.CS2 + 0.4 * torch.eye(3, dtype=E.DT)))
    assert _fourier_gap() > 1e-3


def test_wrong_lift_normalisation_is_caught(monkeypatch):
    orig = E.lift
    monkeypatch.setattr(E, "lift", lambda a: 0.5 * orig(a))
    assert _fourier_gap() > 1e-3


def test_flipped_correction_sign_is_caught(monkeypatch):
    orig = E.entropic_amplitude

    def bad(phi, g_eq, dh, ds_post, u, theta=1e-8, mode="literal"):
        # C enters with the wrong sign: lambda' = 1 + (hs - C)/hh
        lam = orig(phi, g_eq, dh, ds_post, u, theta, mode)
        hh = (dh * dh / g_eq).sum(0)
        corr = (dh * torch.log(g_eq / E._bcast(E.W, g_eq))).sum(0)
        return lam - 2 * corr / hh
    monkeypatch.setattr(E, "entropic_amplitude", bad)
    assert _root_gap() > 5e-2
