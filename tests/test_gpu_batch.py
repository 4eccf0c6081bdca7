"""Batched uneven periodic domains (orientation / anisotropy sweep): the
persistent graph-captured kernel, the per-step batched graph and the 512-style
per-domain launches against the oracle and the exact Fourier recurrence."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from fourier_pin import mode_history

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_2605_01774_gb300 import elbm
    elbm.lib()
    return elbm


def _make(E, table):
    edges = [d["n"] for d in table]
    D6 = np.stack([synth.d6_from_matrix(d["D"]) for d in table])
    h = E.elbm_batch_create(edges, D6)
    phi0 = np.concatenate([synth.batched_phi0(n).ravel() for n in edges]).astype(np.float32)
    return h, phi0, edges


def _split(phi, edges):
    out, o = [], 0
    for n in edges:
        out.append(phi[o:o + n ** 3].reshape(n, n, n))
        o += n ** 3
    return out


def test_small_batch_modes_and_oracle(E):
    table, _ = synth.batched_domains(ndom=10, seed=11, nmin=5, nmax=14)
    h, phi0, edges = _make(E, table)
    res = {}
    for mode in (0, 1, 2):
        E.elbm_batch_init_equilibrium(h, torch.as_tensor(phi0, device="cuda"))
        E.elbm_batch_step(h, 12, mode)
        E.elbm_batch_synchronize(h)
        phi = torch.empty(len(phi0), dtype=torch.float32, device="cuda")
        E.elbm_batch_read_phi(h, phi)
        torch.cuda.synchronize()
        res[mode] = phi.cpu().numpy()
    assert np.array_equal(res[0], res[1])
    assert np.abs(res[0] - res[2]).max() < 1e-6
    for d, (dom, phi) in enumerate(zip(table, _split(res[0], edges))):
        prob = O.Problem.from_tensor(np.zeros(3), dom["D"], theta=3e-4)
        ref = O.run(O.init_equilibrium(synth.batched_phi0(dom["n"]), np.zeros(3)), prob, 12).sum(0).numpy()
        assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-6, d
    g = torch.empty(27 * edges[3] ** 3, dtype=torch.float32, device="cuda")
    E.elbm_batch_read_populations(h, 3, g)
    torch.cuda.synchronize()
    assert abs(g.sum().item() - res[0][sum(n ** 3 for n in edges[:3]):][:edges[3] ** 3].sum()) < 1e-3
    assert E.elbm_batch_fallback_count(h) == 0
    E.elbm_batch_destroy(h)


def test_barrier_timeout_is_reported_and_context_survives(E):
    table, _ = synth.batched_domains(ndom=4, seed=12, nmin=8, nmax=12)
    h, phi0, edges = _make(E, table)
    E.elbm_batch_init_equilibrium(h, torch.as_tensor(phi0, device="cuda"))
    E.elbm_batch_set_wait_limit(h, 2_000_000, extra_arrivals=1)   # a barrier nobody completes
    E.elbm_batch_step(h, 3, 0)
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_batch_synchronize(h)
    assert ei.value.status == 7                                   # ELBM_ERR_TIMEOUT
    E.elbm_batch_set_wait_limit(h, 2_000_000_000, 0)
    E.elbm_batch_init_equilibrium(h, torch.as_tensor(phi0, device="cuda"))
    E.elbm_batch_step(h, 3, 0)
    E.elbm_batch_synchronize(h)
    E.elbm_batch_destroy(h)


def test_full_sweep_exact_recurrence_every_domain(E):
    """512 domains, edges U{16..96} (137 M nodes), 500 steps, persistent graph after
    autotuning: every domain's mode k = 2 pi (1,1,0)/n follows the exact u = 0 recurrence."""
    table, steps = synth.batched_domains()
    h, phi0, edges = _make(E, table)
    E.elbm_batch_init_equilibrium(h, torch.as_tensor(phi0, device="cuda"))
    tile, bps = E.elbm_batch_autotune(h, 2)
    E.elbm_batch_init_equilibrium(h, torch.as_tensor(phi0, device="cuda"))
    E.elbm_batch_step(h, steps, 0)
    E.elbm_batch_synchronize(h)
    info = E.elbm_batch_info(h)
    print("batched: tile", tile, "blocks/SM", bps, "in graph", info["persistent_in_graph"], "nodes",
          info["total_nodes"])
    phi = torch.empty(len(phi0), dtype=torch.float32, device="cuda")
    E.elbm_batch_read_phi(h, phi)
    torch.cuda.synchronize()
    assert E.elbm_batch_fallback_count(h) == 0
    worst = 0.0
    for dom, f in zip(table, _split(phi.cpu().numpy().astype(np.float64), edges)):
        n = dom["n"]
        k = 2 * math.pi * np.array([1.0, 1.0, 0.0]) / n
        S = np.linalg.inv(0.5 * np.eye(3) + 3.0 * dom["D"])
        a0 = np.fft.fftn(synth.batched_phi0(n))[0, 1, 1]
        pred = mode_history(k, S, a0, steps)[-1]
        got = np.fft.fftn(f)[0, 1, 1]
        worst = max(worst, abs(got - pred) / abs(a0))
    print("worst mode error / initial amplitude", worst)
    assert worst < 2e-5
    E.elbm_batch_destroy(h)
