"""Exact Fourier recurrence of the zero-velocity scheme, derived independently
of the oracle (test helper, not part of the oracle).

At u = 0 the stabilizer amplitude is exactly 1 and the post-collision state of
a node depends only on (phi, j):  g*_i = W_i (phi + c_i.(I - S) j / cs2).
Streaming multiplies mode k by exp(-i k.c_i), so (phi_hat, j_hat) evolves by
the 4x4 matrix A(k) = sum_i W_i exp(-i k.c_i) [1; c_i] [1, 3 c_i^T (I - S)].
Velocity set and weights are rebuilt here from the tensor-product definition.
"""
import itertools

import numpy as np

_C = np.array(list(itertools.product((-1, 0, 1), repeat=3)), dtype=float)
_M = (_C != 0).sum(1)
_W = (2.0 / 3.0) ** (3 - _M) * (1.0 / 6.0) ** _M


def amplification(k, S):
    A = np.zeros((4, 4), dtype=complex)
    ImS = np.eye(3) - S
    for i in range(27):
        ph = np.exp(-1j * (_C[i] @ k))
        A += _W[i] * ph * np.outer(np.r_[1.0, _C[i]], np.r_[1.0, 3.0 * (_C[i] @ ImS)])
    return A


def dominant_rate(k, S):
    ev = np.linalg.eigvals(amplification(k, S))
    return -np.log(np.abs(ev[np.argmax(np.abs(ev))]))


def mode_history(k, S, phi_hat0, nsteps):
    A = amplification(k, S)
    v = np.array([phi_hat0, 0, 0, 0], dtype=complex)
    out = []
    for _ in range(nsteps):
        v = A @ v
        out.append(v[0])
    return np.array(out)


# ---- the same recurrence on the two-dimensional set D2Q9 (3 x 3 amplification matrix)
_C2 = np.array(list(itertools.product((-1, 0, 1), repeat=2)), dtype=float)
_M2 = (_C2 != 0).sum(1)
_W2 = (2.0 / 3.0) ** (2 - _M2) * (1.0 / 6.0) ** _M2


def amplification_2d(k, S):
    A = np.zeros((3, 3), dtype=complex)
    ImS = np.eye(2) - S
    for i in range(9):
        ph = np.exp(-1j * (_C2[i] @ k))
        A += _W2[i] * ph * np.outer(np.r_[1.0, _C2[i]], np.r_[1.0, 3.0 * (_C2[i] @ ImS)])
    return A


def dominant_rate_2d(k, S):
    ev = np.linalg.eigvals(amplification_2d(k, S))
    return -np.log(np.abs(ev[np.argmax(np.abs(ev))]))


def mode_history_2d(k, S, phi_hat0, nsteps):
    A = amplification_2d(k, S)
    v = np.array([phi_hat0, 0, 0], dtype=complex)
    out = []
    for _ in range(nsteps):
        v = A @ v
        out.append(v[0])
    return np.array(out)
