"""Pin of the oracle's misfit gradient (oracle.adjoint.misfit_gradient): reverse-mode
differentiation of the literal program must equal central finite differences of the misfit
J(theta) = 1/2 sum_{t in obs} sum_x (phi_t - phi*_t)^2 itself, on a 6^3 box with u != 0 (the
entropic amplitude is active) and the positivity fallback inactive, with and without
checkpointed segments.  Errors are relative to the difference quotient, or to 1e-3 of the
largest gradient entry where the quotient is smaller than that."""
import numpy as np
import pytest
import torch

import oracle.adjoint as A
import synth

STEPS, OBS, U = 6, (3, 6), (0.02, 0.01, -0.015)


def _problem():
    dims = (6, 6, 6)
    g = synth.rng(21)
    th_true = np.empty((6,) + dims)
    for k, base in enumerate((1e-2, 1e-3, 1e-4)):
        th_true[k] = np.log(base) + 0.3 * synth.smooth_noise(dims, g, 1.5)
    for k in range(3):
        th_true[3 + k] = g.uniform(0, 2 * np.pi) + 0.5 * synth.smooth_noise(dims, g, 1.5)
    th0 = th_true + 0.1 * np.stack([synth.smooth_noise(dims, g, 1.0) for _ in range(6)])
    phi0 = 1.0 + 0.5 * synth.gaussian(dims, (2.5, 2.5, 2.5), 1.5)
    targets = A.forward_snapshots(th_true, phi0, U, STEPS, OBS)
    return th0, phi0, targets


def _central(th0, p, h, phi0, targets):
    tp, tm = th0.copy(), th0.copy()
    tp[p] += h
    tm[p] -= h
    Jp = float(A.misfit(torch.as_tensor(tp), phi0, U, STEPS, OBS, targets)[0])
    Jm = float(A.misfit(torch.as_tensor(tm), phi0, U, STEPS, OBS, targets)[0])
    return (Jp - Jm) / (2 * h)


def _fd_errors(segment=None, h=4e-3):
    th0, phi0, targets = _problem()
    J, grad, nfb = A.misfit_gradient(th0, phi0, U, STEPS, OBS, targets, segment=segment)
    assert nfb == 0
    rng = np.random.default_rng(7)
    picks = [(int(rng.integers(6)),) + tuple(int(v) for v in rng.integers(0, 6, 3)) for _ in range(12)]
    picks += [(k, 2, 3, 2) for k in range(6)]            # every parameter kind near the plume centre
    errs = []
    for p in picks:
        # Richardson extrapolation of two central differences: the O(h^2) error term cancels
        fd = (4.0 * _central(th0, p, h / 2, phi0, targets) - _central(th0, p, h, phi0, targets)) / 3.0
        g = float(grad[p])
        errs.append(abs(g - fd) / max(abs(fd), 1e-3 * float(grad.abs().max())))
    return max(errs), J


@pytest.mark.parametrize("segment", [None, 2])
def test_misfit_gradient_matches_central_differences(segment):
    err, J = _fd_errors(segment)
    assert J > 0
    assert err < 1e-6, err
