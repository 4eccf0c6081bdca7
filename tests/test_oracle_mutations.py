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


# ---- pins of the tensor parametrisation, the entropy diagnostic and the misfit gradient

def _table1_gap():
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
    blk = gold["table1_gaussian_tensor_targets"]
    worst = 0.0
    for row in blk["rows"]:
        th = torch.tensor([math.log(v) for v in row["d"]] + [math.radians(a) for a in blk["euler_deg"]],
                          dtype=torch.float64)
        D = O.tensor_from_params(th)
        d6 = torch.stack([D[0, 0], D[0, 1], D[0, 2], D[1, 1], D[1, 2], D[2, 2]]).numpy() * 1e3
        worst = max(worst, float(np.abs(d6 - np.asarray(row["target_1e3"])).max()))
    return worst


def _entropy_gap():
    phi = np.random.default_rng(3).uniform(0.05, 2.0, (3, 4, 5))
    g = O.equilibrium(torch.as_tensor(phi), torch.zeros(3, dtype=torch.float64))
    return abs(O.diagnostics(g)["entropy"] - float(np.sum(phi * np.log(phi)))) / abs(float(np.sum(phi * np.log(phi))))


def test_unmutated_baseline_params_entropy():
    assert _table1_gap() < 5.5e-5
    assert _entropy_gap() < 1e-13


def test_transposed_rotation_is_caught(monkeypatch):
    orig = E.rotation_zyz
    monkeypatch.setattr(E, "rotation_zyz", lambda a, b, c: orig(a, b, c).transpose(-1, -2))
    assert _table1_gap() > 1e-3


def test_swapped_euler_order_is_caught(monkeypatch):
    orig = E.rotation_zyz
    monkeypatch.setattr(E, "rotation_zyz", lambda a, b, c: orig(c, b, a))
    assert _table1_gap() > 1e-3


def test_entropy_without_weights_is_caught(monkeypatch):
    # H computed as sum g ln g (the W_i dropped from Eq. method-entropy)
    monkeypatch.setattr(E, "W", torch.ones(27, dtype=torch.float64))
    assert _entropy_gap() > 1e-3


def test_gradient_lost_through_checkpoints_is_caught(monkeypatch):
    """Re-entrant checkpointing computes gradients only for a segment's tensor inputs, so the
    dependence on theta through the relaxation matrix captured by the segment is dropped."""
    import oracle.adjoint as A
    from test_oracle_adjoint import _fd_errors
    from torch.utils.checkpoint import checkpoint as ck
    monkeypatch.setattr(A, "checkpoint", lambda f, *a, **k: ck(f, *a, use_reentrant=True))
    try:
        err, _ = _fd_errors(segment=2)
    except RuntimeError:          # nothing left that requires a gradient
        err = float("inf")
    assert err > 1e-3


# ---- D2Q9 oracle

def _fourier_gap_2d():
    import oracle.d2q9 as O2
    from fourier_pin import mode_history_2d
    nx, ny, m = 9, 7, (2, -1)
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    k = 2 * math.pi * np.array([m[0] / nx, m[1] / ny])
    phi0 = 1.0 + 0.1 * np.sin(k[0] * x + k[1] * y)
    a = 0.7
    R = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    D = R @ np.diag([0.05, 0.005]) @ R.T
    prob = O2.Problem.from_tensor((0.0, 0.0), D)
    idx = (m[1] % ny, m[0] % nx)
    hist = []
    O2.run(O2.init_equilibrium(phi0, (0.0, 0.0)), prob, 20,
           callback=lambda n, g: hist.append(np.fft.fft2(g.sum(0).numpy())[idx]))
    S = np.linalg.inv(0.5 * np.eye(2) + 3.0 * D)
    pred = mode_history_2d(k, S, np.fft.fft2(phi0)[idx], 20)
    return np.max(np.abs(np.array(hist) - pred)) / abs(np.fft.fft2(phi0)[idx])


def test_unmutated_baseline_2d():
    assert _fourier_gap_2d() < 1e-12


def test_2d_wrong_lift_normalisation_is_caught(monkeypatch):
    import oracle.d2q9 as O2
    orig = O2.lift
    monkeypatch.setattr(O2, "lift", lambda a: 0.5 * orig(a))
    assert _fourier_gap_2d() > 1e-3


def test_2d_transposed_streaming_axes_is_caught(monkeypatch):
    """Streaming that rolls x along the y axis and y along the x axis (an oblique mode on a
    non-square grid sees it)."""
    import oracle.d2q9 as O2

    def bad(gp):
        out = torch.empty_like(gp)
        for i, (cx, cy) in enumerate(O2.C_INT):
            out[i] = torch.roll(gp[i], shifts=(cx, cy), dims=(0, 1))
        return out
    monkeypatch.setattr(O2, "stream", bad)
    assert _fourier_gap_2d() > 1e-3
