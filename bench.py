"""Throughput of the fused ELBM-ADE step on the advected anisotropic Gaussian
plume (256^3 periodic, u = (0.05, 0.03, 0.02), D = R diag(0.1, 1e-3, 1e-5) R^T,
sigma0 = 8), in MLUPS and as a fraction of the measured HBM bandwidth.

One step = one collide-stream pass over the whole lattice.  The headline is the
chosen form: by default FP32 arithmetic and storage, which on this workload is both
the fastest form on GB300 (HBM-bound) and the most accurate of the FP32-arithmetic
forms.  The FP16 and BF16 deviation storages (half the bytes, but issue-bound on
the decode/encode and the positivity fallback) and FP64 are measured beside it,
each with its relative L2 error of phi against the FP64 form after a fixed number
of steps (the FP64 form itself matches the FP64 oracle to 1e-12 in the parity
tests) and its speedup over the plain FP32 form.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank steps its own replica of the
lattice (the method has no data-path exchange for independent problems), and
`value` is the node updates of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "ELBM-ADE MLUPS & % HBM roofline, chosen vs plain form at stated L2 error"
UNIT = "MLUPS"
KERNEL_NAME = {1: "k_step", 2: "k_step_rows", 3: "k_step_pipe"}
F64_FLOPS_PER_NODE = 706   # mean of the two launches in profiles/k_step_fp64_plume128_flops.md
BYTES_PER_NODE = {"f64": 27 * 8 * 2, "f32": 27 * 4 * 2, "f16dev": (27 * 2 + 4) * 2, "bf16dev": (27 * 2 + 4) * 2}
WORKLOAD = ("advected anisotropic Gaussian plume 256^3 periodic, u=(0.05,0.03,0.02), "
            "D=R diag(0.1,1e-3,1e-5) R^T (seeded ZYZ, seed 2), sigma0=8")
KERNEL_SOURCES = ["collide.cuh", "eqlog.cuh", "storage.cuh", "pull.cuh", "step.cu", "step_rows.cu", "bulk.cuh",
                  "lattice.cuh"]
THETA = 3e-4   # stabilizer guard used by every form, so the forms differ only in arithmetic and storage


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2605_01774_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
    return 6800.0, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


def ncu_traffic(form: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on the current kernel."""
    p = os.path.join(ROOT, "profiles", "step_traffic.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        parts = line.split()
        if len(parts) == 2 and not line.startswith("#"):
            vals[parts[0]] = parts[1]
    if vals.get("kernel_hash") != kernel_hash() or form not in vals:
        return None
    return float(vals[form])


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons sampled every 10 ms, started a moment before the
    timed region; the summary keeps the samples whose timestamps fall inside the region (host
    clock from just before the first timed launch to just after the last one completed), so that
    a timed region of a few milliseconds still has its own samples and idle samples around it do
    not count."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    LEAD_S = 0.3   # nvidia-smi's start-up before the first sample

    def __init__(self, device: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.device = device
        self.p = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "10", "-i", str(self.device)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
            time.sleep(self.LEAD_S)
        except (OSError, FileNotFoundError):
            self.p = None
        return self

    def start(self):
        """Mark the start of the timed region (call just before its first launch)."""
        self.t0 = time.time()

    def stop(self):
        """Mark its end (call once its last launch has completed)."""
        self.t1 = time.time()

    def __exit__(self, *a):
        if self.p is not None:
            time.sleep(0.03)   # let the sample that follows the region land
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        import datetime
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        inside = [r for r in rows if self.t0 is not None and self.t1 is not None and self.t0 <= r[0] <= self.t1]
        note = None
        if not inside and rows and self.t0 is not None and self.t1 is not None:
            # a region shorter than the sampling interval: the sample nearest to it, marked as such
            near = min(rows, key=lambda r: max(self.t0 - r[0], r[0] - self.t1, 0.0))
            note = f"no sample inside the {1e3 * (self.t1 - self.t0):.1f} ms region; nearest " \
                   f"{1e3 * max(self.t0 - near[0], near[0] - self.t1, 0.0):.1f} ms from it"
            inside = [near]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in inside for k in range(4) if r[3][k].lower().startswith("active")})
        out = {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
               "reasons": reasons, "samples": len(inside) if note is None else 0,
               "interval_ms": 10, "region_ms": round(1e3 * (self.t1 - self.t0), 2)}
        if note:
            out["note"] = note
        return out


def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(v: float, dist, device=None) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v: float, dist, device=None) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------- our arm
def run_ours(args, rank, world, local, dist):
    import torch

    from paper_2605_01774_gb300 import elbm as E

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    E.lib()
    wl = synth.gaussian_plume(n=args.size, dims=args.dims if args.only else None)
    D6 = synth.d6_from_matrix(wl.D)
    N = int(np.prod(wl.dims))
    stream = torch.cuda.Stream(device=dev)
    phi0 = torch.as_tensor(wl.phi0, dtype=torch.float32, device=dev)

    def make(prec):
        lat = E.Lattice(wl.dims, prec, stream=stream)
        E.elbm_set_tensor_uniform(lat.h, D6)
        E.elbm_set_velocity_uniform(lat.h, wl.u)
        E.elbm_set_params(lat.h, theta=THETA)
        E.elbm_set_step_kernel(lat.h, args.step_kernel)
        stream.wait_stream(torch.cuda.current_stream(dev))
        E.elbm_init_equilibrium(lat.h, phi0)
        return lat

    def timed(lat, K, W, sample_clocks=False):
        E.elbm_step(lat.h, W)
        stream.synchronize()
        barrier(dist)
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.__enter__()
            sampler.start()
        ev0.record(stream)
        E.elbm_step(lat.h, K)
        ev1.record(stream)
        ev1.synchronize()
        if sampler:
            sampler.stop()
            sampler.__exit__(None, None, None)
        torch.cuda.synchronize(dev)
        barrier(dist)
        ms = ev0.elapsed_time(ev1)
        return ms, (sampler.summary() if sampler else None)

    if args.d2_only:
        # one D2Q9 form on the 4096^2 field workload, no comparison (the command profiled by ncu)
        return run_d2q9(args, E, dev, stream, dist, world, forms=(args.d2_only,))

    if args.only and args.workload == "heterogeneous":
        # the 384^3 two-phase porous workload (per-node tensor field, Gaussian source, Dirichlet
        # x faces, u = 0): a parity-test configuration, timed here for one form
        hw = synth.heterogeneous(n=args.size if args.size != 256 else 384, dims=args.dims)
        Nh = int(np.prod(hw.dims))
        lat = E.Lattice(hw.dims, args.only, bc=hw.dirichlet_x, stream=stream)
        E.elbm_set_tensor_field(lat.h, torch.as_tensor(hw.D6_field, dtype=torch.float32, device=dev))
        E.elbm_set_source(lat.h, torch.as_tensor(hw.source, dtype=torch.float32, device=dev))
        E.elbm_set_params(lat.h, theta=THETA)
        E.elbm_set_step_kernel(lat.h, args.step_kernel)
        stream.wait_stream(torch.cuda.current_stream(dev))
        E.elbm_init_equilibrium(lat.h, torch.as_tensor(hw.phi0, dtype=torch.float32, device=dev))
        ms, _ = timed(lat, args.steps, args.warmup)
        kern = KERNEL_NAME[E.elbm_get_step_kernel(lat.h)]
        lat.close()
        # + tensor field (6 values in the arithmetic type) and the FP32 source plane
        bpn = BYTES_PER_NODE[args.only] + (48 if args.only == "f64" else 24) + 4
        peak, _ = measured_peaks()
        return {"only": args.only, "workload": "heterogeneous", "nodes": Nh, "kernel": kern,
                "ms_per_step": ms / args.steps, "mlups": Nh * args.steps / (ms * 1e-3) / 1e6,
                "bytes_per_node": bpn, "hbm_frac_of_measured": bpn * Nh / (ms / args.steps * 1e-3) / 1e9 / peak}

    if args.only:
        # one form, timing only (the command profiled by ncu)
        lat = make(args.only)
        ms, _ = timed(lat, args.steps, args.warmup)
        kern = KERNEL_NAME[E.elbm_get_step_kernel(lat.h)]
        lat.close()
        return {"only": args.only, "nodes": N, "kernel": kern, "ms_per_step": ms / args.steps,
                "mlups": N * args.steps / (ms * 1e-3) / 1e6}

    forms = {}
    headline = args.form
    order = [headline] + [f for f in ("f32", "bf16dev", "f16dev") if f != headline]
    clocks = None
    late = None
    for prec in order:
        lat = make(prec)
        ms, ck = timed(lat, args.steps, args.warmup, sample_clocks=(prec == headline))
        if prec == headline:
            clocks = ck
        d = E.elbm_reduce(lat.h, allow_nonfinite=True)
        proj = E.elbm_storage_projections(lat.h)
        kern = KERNEL_NAME[E.elbm_get_step_kernel(lat.h)]
        if prec == headline and args.late_window > 0:
            late = late_window(args, E, lat, stream, dev, dist, N, d["n_fallback"], local)
        lat.close()
        ms_max = max_over_ranks(ms, dist, dev)
        forms[prec] = dict(ms_per_step=ms_max / args.steps,
                           mlups=world * N * args.steps / (ms_max * 1e-3) / 1e6,
                           bytes_per_node=BYTES_PER_NODE[prec], n_fallback=d["n_fallback"],
                           n_projected=proj, finite=d["status"] == 0, kernel=kern)
    # FP64: ALU-bound on this part; fewer steps keep the run short
    k64 = max(10, min(args.steps, 200))
    lat = make("f64")
    ms, _ = timed(lat, k64, min(args.warmup, 3))
    d = E.elbm_reduce(lat.h, allow_nonfinite=True)
    lat.close()
    ms = max_over_ranks(ms, dist, dev)
    forms["f64"] = dict(ms_per_step=ms / k64, mlups=world * N * k64 / (ms * 1e-3) / 1e6,
                        bytes_per_node=BYTES_PER_NODE["f64"], steps=k64, n_fallback=d["n_fallback"])
    # FP64 is bound by FP64 FMA throughput on this part: its arithmetic roofline against the
    # measured FMA peak, with the per-node flop count from the committed ncu summary
    peak64 = E.elbm_fma_peak("f64")
    achieved64 = F64_FLOPS_PER_NODE * forms["f64"]["mlups"] * 1e6 / world
    forms["f64"]["alu_roofline"] = {"bound": "alu", "unit": "TFLOP/s", "peak": peak64 / 1e12,
                                    "achieved": achieved64 / 1e12, "frac": achieved64 / peak64,
                                    "flops_per_node": F64_FLOPS_PER_NODE,
                                    "source": "peak: elbm_fma_peak (measured now); flops per node: "
                                              "profiles/k_step_fp64_plume128_flops.md"}

    # accuracy: phi after `ek` steps of each form vs the FP64 form (parity-tested against the oracle)
    ek = args.err_steps
    phis = {}
    for prec in ["f64"] + order:
        lat = make(prec)
        E.elbm_step(lat.h, ek)
        out = torch.empty(wl.dims[::-1], dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            E.elbm_read_moments(lat.h, out)
        stream.synchronize()
        phis[prec] = out
        lat.close()
    ref = phis["f64"]
    for prec in order:
        forms[prec]["rel_l2_phi_vs_fp64"] = float(torch.linalg.vector_norm(phis[prec] - ref) /
                                                  torch.linalg.vector_norm(ref))
        forms[prec]["rel_linf_phi_vs_fp64"] = float((phis[prec] - ref).abs().max() / ref.abs().max())
    del phis, ref

    # end to end through the C ABI with host buffers: upload phi0, K steps, read phi back
    host_phi0 = torch.as_tensor(wl.phi0, dtype=torch.float32).pin_memory()
    host_out = torch.empty(wl.dims[::-1], dtype=torch.float32).pin_memory()
    lat = E.Lattice(wl.dims, headline, stream=stream)
    E.elbm_set_tensor_uniform(lat.h, D6)
    E.elbm_set_velocity_uniform(lat.h, wl.u)
    E.elbm_set_step_kernel(lat.h, args.step_kernel)
    E.elbm_init_equilibrium(lat.h, host_phi0)
    E.elbm_step(lat.h, args.warmup)
    stream.synchronize()
    barrier(dist)
    t0 = time.perf_counter()
    E.elbm_init_equilibrium(lat.h, host_phi0)
    E.elbm_step(lat.h, args.steps)
    E.elbm_read_moments(lat.h, host_out)
    mass = E.elbm_reduce(lat.h, allow_nonfinite=True)["mass"]
    t_e2e = time.perf_counter() - t0
    lat.close()
    t_e2e = max_over_ranks(t_e2e, dist, dev)
    e2e = dict(value=world * N * args.steps / t_e2e / 1e6, unit=UNIT,
               h2d_bytes_per_step=N * 4 / args.steps, d2h_bytes_per_step=(N * 4 + 8 * 4) / args.steps,
               final_mass=mass)

    batched = None if args.batched_steps <= 0 else run_batched(args, E, dev, dist, world)
    extra = {}
    if not args.skip_extra:
        extra["heterogeneous"] = run_heterogeneous(args, E, dev, stream, dist, world)
        extra["adjoint"] = run_adjoint(args, E, dev, dist, world)
        extra["d2q9"] = run_d2q9(args, E, dev, stream, dist, world)

    if rank != 0:
        return None
    peak, peak_src = measured_peaks()
    hf = forms[headline]
    achieved = hf["bytes_per_node"] * N / (hf["ms_per_step"] * 1e-3) / 1e9
    traffic = ncu_traffic(headline)
    for prec in order + ["f64"]:
        f = forms[prec]
        f["achieved_gbs"] = f["bytes_per_node"] * N / (f["ms_per_step"] * 1e-3) / 1e9
        f["hbm_frac_of_measured"] = f["achieved_gbs"] / peak
    line = {
        "metric": METRIC, "value": hf["mlups"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": hf["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f16dev": "f32 compute, f16 deviation storage",
                  "bf16dev": "f32 compute, bf16 deviation storage"}[headline], "data": "synthetic",
        "config": {"workload": WORKLOAD, "nodes": N, "form": headline, "plain_form": "f32",
                   "l2_flush": "inputs larger than L2: %.2f GB per population buffer" %
                               (hf["bytes_per_node"] / 2 * N / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "err_steps": ek, "step_kernel": args.step_kernel},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes_per_node": hf["bytes_per_node"], "kernel": hf["kernel"]},
        "forms": forms,
        "chosen_vs_plain_speedup": hf["mlups"] / forms["f32"]["mlups"],
        "vs_plain_speedup": {p: forms[p]["mlups"] / forms["f32"]["mlups"] for p in order + ["f64"]},
        "e2e": e2e,
        "late_window": late,
        "batched": batched,
        **extra,
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    return line


def late_window(args, E, lat, stream, dev, dist, N, fb_so_far, local):
    """The headline form's rate late in the run: the same lattice advanced (untimed) to step
    `late_start`, then `late_window` steps timed with CUDA events on the launching stream, with
    the fallback fraction of those steps and the SM clocks sampled meanwhile."""
    import torch
    done = E.elbm_get_step(lat.h)
    if args.late_start > done:
        E.elbm_step(lat.h, args.late_start - done)
    fb0 = E.elbm_reduce(lat.h, allow_nonfinite=True)["n_fallback"]
    stream.synchronize()
    barrier(dist)
    sampler = ClockSampler(local)
    sampler.__enter__()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.start()
    ev0.record(stream)
    E.elbm_step(lat.h, args.late_window)
    ev1.record(stream)
    ev1.synchronize()
    sampler.stop()
    sampler.__exit__(None, None, None)
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev) / args.late_window
    fb1 = E.elbm_reduce(lat.h, allow_nonfinite=True)["n_fallback"]
    peak, _ = measured_peaks()
    bpn = BYTES_PER_NODE[args.form]
    return {"steps": [args.late_start, args.late_start + args.late_window], "ms_per_step": ms,
            "mlups": N / (ms * 1e-3) / 1e6, "hbm_frac_of_measured": bpn * N / (ms * 1e-3) / 1e9 / peak,
            "fallback_node_fraction": (fb1 - fb0) / (args.late_window * N),
            "fallback_node_fraction_timed_window": fb_so_far / ((args.steps + args.warmup) * N),
            "clocks": sampler.summary()}


def _time_steps(E, step_fn, K, stream):
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    step_fn(K)
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1) / K


def run_heterogeneous(args, E, dev, stream, dist, world):
    """Two-phase porous transport at 384^3 (per-node tensor field from a seeded rotation field
    and porous mask, Gaussian source, Dirichlet x faces at the shifted values 2 and 1, u = 0):
    ms/step, MLUPS and HBM fraction per form (bytes: populations read and written, the per-node
    T field and the FP32 source plane), and the relative L2 error of phi against the FP64 form
    after `het_err_steps` steps from the same start.  The run to steady state of this workload
    is checked on a 48^3 twin in the tests (about 2e5 steps there; 1.5e6 at 384^3)."""
    import torch
    hw = synth.heterogeneous(n=args.het_size)
    Nh = int(np.prod(hw.dims))
    D6 = torch.as_tensor(hw.D6_field, dtype=torch.float32, device=dev)
    src = torch.as_tensor(hw.source, dtype=torch.float32, device=dev)
    phi0 = torch.as_tensor(hw.phi0, dtype=torch.float32, device=dev)
    del hw.D6_field
    peak, _ = measured_peaks()

    def make(prec):
        lat = E.Lattice(hw.dims, prec, bc=hw.dirichlet_x, stream=stream)
        E.elbm_set_tensor_field(lat.h, D6)
        E.elbm_set_source(lat.h, src)
        E.elbm_set_params(lat.h, theta=THETA)
        stream.wait_stream(torch.cuda.current_stream(dev))
        E.elbm_init_equilibrium(lat.h, phi0)
        return lat

    out = {"workload": "two-phase porous 384^3, per-node tensor field, Gaussian source, Dirichlet x (2, 1), u = 0",
           "nodes": Nh * world, "err_steps": args.het_err_steps, "forms": {}}
    phis = {}
    for prec in ("f64", "f32", "f16dev", "bf16dev"):
        lat = make(prec)
        E.elbm_step(lat.h, args.het_err_steps)
        ph = torch.empty(hw.dims[::-1], dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            E.elbm_read_moments(lat.h, ph)
        E.elbm_step(lat.h, 3)
        stream.synchronize()
        barrier(dist)
        K = args.het_steps if prec != "f64" else max(5, args.het_steps // 10)
        ms = max_over_ranks(_time_steps(E, lambda k: E.elbm_step(lat.h, k), K, stream), dist, dev)
        fb = E.elbm_reduce(lat.h, allow_nonfinite=True)["n_fallback"]
        bpn = BYTES_PER_NODE[prec] + (48 if prec == "f64" else 24) + 4
        mlups = world * Nh / (ms * 1e-3) / 1e6
        out["forms"][prec] = {"kernel": KERNEL_NAME[E.elbm_get_step_kernel(lat.h)], "ms_per_step": ms, "mlups": mlups,
                              "bytes_per_node": bpn, "hbm_frac_of_measured": bpn * mlups / world * 1e6 / 1e9 / peak,
                              "n_fallback": fb}
        lat.close()
        phis[prec] = ph
    ref = phis["f64"]
    for prec in ("f32", "f16dev", "bf16dev"):
        out["forms"][prec]["rel_l2_phi_vs_fp64"] = float(torch.linalg.vector_norm(phis[prec] - ref) /
                                                         torch.linalg.vector_norm(ref))
    f32 = out["forms"]["f32"]["mlups"]
    out["vs_plain_speedup"] = {p: out["forms"][p]["mlups"] / f32 for p in out["forms"]}
    return out


def run_adjoint(args, E, dev, dist, world):
    """Inverse problem on a 64^3 box, FP32: per-node (ln d, ZYZ angles) field, u = (0.02, 0, 0),
    500 steps, misfit against snapshots at 250 and 500 from the true field, checkpoints every
    50 steps.  Times the forward sweep alone (the misfit) and the full gradient (forward sweep,
    then per 50-step segment a recomputation and the reverse sweep of hand-written
    vector-Jacobian products); the reverse rate is derived as (gradient - 2 forward) / steps.
    Bytes per node-update: forward 240 (populations in and out, the FP32 T field), one VJP step
    444 (forward populations, adjoint populations in and out, T, the FP64 T accumulator read and
    written).  At 64^3 the working set (63 MB per forward step) fits in L2, so these are rates,
    not HBM-roofline fractions."""
    import torch
    p = synth.adjoint_problem(n=args.adj_size, steps=args.adj_steps, obs=(args.adj_steps // 2, args.adj_steps))
    dims, N = p["dims"], int(np.prod(p["dims"]))
    th_true = torch.as_tensor(p["theta_true"], dtype=torch.float32, device=dev)
    th0 = torch.as_tensor(p["theta0"], dtype=torch.float32, device=dev)
    phi0 = torch.as_tensor(p["phi0"], dtype=torch.float32, device=dev)
    # targets: phi of the true field at the observation steps, from the single-lattice path
    lat = E.Lattice(dims, "f32")
    E.elbm_set_tensor_params_field(lat.h, th_true)
    E.elbm_set_velocity_uniform(lat.h, p["u"])
    E.elbm_set_params(lat.h, theta=1e-8)
    E.elbm_init_equilibrium(lat.h, phi0)
    tg = torch.empty((2,) + dims[::-1], dtype=torch.float32, device=dev)
    t = 0
    for o, ts in enumerate(p["obs"]):
        E.elbm_step(lat.h, ts - t)
        t = ts
        E.elbm_read_moments(lat.h, tg[o])
    torch.cuda.synchronize()
    lat.close()
    h = E.elbm_adjoint_create(dims, "f32")
    E.elbm_adjoint_configure(h, p["u"], 1e-8, 50)
    grad = torch.empty((6,) + dims[::-1], dtype=torch.float32, device=dev)
    E.elbm_adjoint_misfit(h, th0, phi0, p["steps"], p["obs"], tg, grad)       # warm-up
    barrier(dist)
    t0 = time.perf_counter()
    J, _ = E.elbm_adjoint_misfit(h, th0, phi0, p["steps"], p["obs"], tg)[:2]
    t_fwd = max_over_ranks(time.perf_counter() - t0, dist, dev)
    t0 = time.perf_counter()
    res = E.elbm_adjoint_misfit(h, th0, phi0, p["steps"], p["obs"], tg, grad)
    t_grad = max_over_ranks(time.perf_counter() - t0, dist, dev)
    E.elbm_adjoint_destroy(h)
    S = p["steps"]
    fwd = t_fwd * 1e3 / S
    rev = max(t_grad - 2 * t_fwd, 1e-9) * 1e3 / S
    return {"workload": "64^3 inverse problem, FP32, 500 steps, obs 250/500, checkpoints every 50",
            "nodes": N * world, "steps": S, "J": float(J), "n_fallback": int(res[-1]),
            "forward_ms_per_step": fwd, "forward_mlups": world * N / (fwd * 1e-3) / 1e6,
            "forward_bytes_per_node": 240, "forward_gbs": 240 * N / (fwd * 1e-3) / 1e9,
            "gradient_ms_per_step": t_grad * 1e3 / S, "reverse_ms_per_step": rev,
            "reverse_mlups": world * N / (rev * 1e-3) / 1e6, "reverse_bytes_per_node": 444,
            "reverse_gbs": 444 * N / (rev * 1e-3) / 1e9,
            "note": "host wall clock per call (synchronous API); 63 MB working set is L2-resident"}


def run_d2q9(args, E, dev, stream, dist, world, forms=("f64", "f32")):
    """D2Q9 (Section 2.1's second velocity set) on a 4096^2 periodic box with channel-shaped
    per-node velocity and tensor fields (Section 4.1's shape): ms/step, MLUPS, bytes per node
    (9 populations read and written, the per-node T field and the FP32 velocity field), HBM
    fraction, and phi after `d2_err_steps` steps against the FP64 form."""
    import torch
    n = args.d2_size
    uf, D3, phi0 = synth.channel2d(n, n, 11)
    uf = torch.as_tensor(uf, dtype=torch.float32, device=dev)
    D3 = torch.as_tensor(D3, dtype=torch.float32, device=dev)
    phi0 = torch.as_tensor(phi0, dtype=torch.float32, device=dev)
    peak, _ = measured_peaks()
    out = {"workload": f"D2Q9 {n}x{n} periodic, per-node velocity and tensor fields", "nodes": n * n * world,
           "forms": {}}
    phis = {}
    for prec in forms:
        lat = E.Lattice2D((n, n), prec, stream=stream)
        E.elbm2d_set_tensor_field(lat.h, D3)
        E.elbm2d_set_velocity_field(lat.h, uf)
        E.elbm2d_set_params(lat.h, theta=THETA)
        stream.wait_stream(torch.cuda.current_stream(dev))
        E.elbm2d_init_equilibrium(lat.h, phi0)
        E.elbm2d_step(lat.h, args.d2_err_steps)
        ph = torch.empty((n, n), dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            E.elbm2d_read_moments(lat.h, ph)
        stream.synchronize()
        barrier(dist)
        ms = max_over_ranks(_time_steps(E, lambda k: E.elbm2d_step(lat.h, k), args.d2_steps, stream), dist, dev)
        es = 8 if prec == "f64" else 4
        bpn = 2 * 9 * es + 3 * es + 8
        mlups = world * n * n / (ms * 1e-3) / 1e6
        out["forms"][prec] = {"ms_per_step": ms, "mlups": mlups, "bytes_per_node": bpn,
                              "hbm_frac_of_measured": bpn * mlups / world * 1e6 / 1e9 / peak,
                              "n_fallback": E.elbm2d_reduce(lat.h, allow_nonfinite=True)["n_fallback"]}
        lat.close()
        phis[prec] = ph
    if "f64" in phis and "f32" in phis:
        out["forms"]["f32"]["rel_l2_phi_vs_fp64"] = float(torch.linalg.vector_norm(phis["f32"] - phis["f64"]) /
                                                          torch.linalg.vector_norm(phis["f64"]))
    out["err_steps"] = args.d2_err_steps
    return out


def shard(items, rank, world):
    """Round-robin share of independent units for one rank (every unit exactly once)."""
    return items[rank::world]


def run_batched(args, E, dev, dist, world):
    """Orientation / anisotropy sweep: 512 periodic domains, edges U{16..96} (seed 4),
    FP32, u = 0; persistent graph-captured kernel (autotuned) vs one batched launch per
    step in a graph vs one plain launch per domain per step.  With several ranks the
    domains are shared round-robin (independent problems: no data-path collective)."""
    import torch
    table, _ = synth.batched_domains()
    rank = dist.get_rank() if dist is not None else 0
    table = shard(table, rank, world)
    edges = [d["n"] for d in table]
    D6 = np.stack([synth.d6_from_matrix(d["D"]) for d in table])
    phi0 = torch.as_tensor(np.concatenate([synth.batched_phi0(n).ravel() for n in edges]).astype(np.float32),
                           device=dev)
    h = E.elbm_batch_create(edges, D6)
    E.elbm_batch_init_equilibrium(h, phi0)
    tile, bps = E.elbm_batch_autotune(h, 2)
    total = E.elbm_batch_info(h)["total_nodes"]
    all_nodes = sum_over_ranks(float(total), dist, dev)
    out = {"domains": len(synth.batched_domains()[0]), "nodes": int(all_nodes), "steps": args.batched_steps,
           "tile": tile,
           "blocks_per_sm": bps, "bytes_per_node": BYTES_PER_NODE["f32"]}
    peak, _ = measured_peaks()
    for mode, name in ((0, "persistent_graph"), (1, "per_step_graph"), (2, "per_domain_launches")):
        E.elbm_batch_init_equilibrium(h, phi0)
        E.elbm_batch_step(h, 2, mode)
        E.elbm_batch_synchronize(h)
        barrier(dist)
        t0 = time.perf_counter()
        E.elbm_batch_step(h, args.batched_steps, mode)
        E.elbm_batch_synchronize(h)
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        mlups = all_nodes * args.batched_steps / dt / 1e6
        out[name] = {"ms_per_step": dt * 1e3 / args.batched_steps, "mlups": mlups,
                     "hbm_frac_of_measured": mlups * 1e6 * BYTES_PER_NODE["f32"] / 1e9 / peak}
    out["persistent_in_graph"] = E.elbm_batch_info(h)["persistent_in_graph"]
    out["persistent_vs_per_domain_speedup"] = out["persistent_graph"]["mlups"] / out["per_domain_launches"]["mlups"]
    E.elbm_batch_destroy(h)
    return out


# ------------------------------------------------------------------------ oracle arm
def oracle_sample(n=40):
    """The bench workload's physics (u, D, sigma0) on a bounded n^3 periodic sample."""
    return synth.gaussian_plume(n=n)


def cpu_model() -> str:
    """Host CPU model: lscpu's model name (Arm hosts report the core, e.g. Neoverse-V2), else
    /proc/cpuinfo's, else the machine type; with the vendor where lscpu gives one."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        info = {}
        for line in out.splitlines():
            if ":" in line:
                k, v = line.split(":", 1)
                info.setdefault(k.strip().lower(), v.strip())
        if info.get("model name"):
            vendor = info.get("vendor id", "")
            return (vendor + " " if vendor and vendor not in info["model name"] else "") + info["model name"]
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _oracle_rate(args, seconds):
    import oracle as O
    wl = oracle_sample(args.cpu_sample)
    prob = O.Problem.from_tensor(wl.u, wl.D, theta=3e-4, lam_mode="literal")
    g = O.init_equilibrium(wl.phi0, wl.u)
    g = O.step(g, prob, 0)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        g = O.step(g, prob, n)
        n += 1
    dt = time.perf_counter() - t0
    return int(np.prod(wl.dims)) * n / dt / 1e6, n, wl.dims


def cpu_baseline(args, seconds=15.0):
    """The FP64 oracle on the host cores (all torch threads), then on one thread."""
    import torch
    threads = torch.get_num_threads()
    v, n, dims = _oracle_rate(args, seconds)
    torch.set_num_threads(1)
    try:
        v1, n1, _ = _oracle_rate(args, seconds / 2)
    finally:
        torch.set_num_threads(threads)
    return {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} steps of the bench physics on a {dims[0]}^3 periodic box (FP64, torch CPU)",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "single_thread": {"value": v1, "unit": UNIT, "threads": 1, "sample": f"{n1} steps, same box"}}


def run_reference(args, rank, world, dist):
    import torch

    import oracle as O
    if rank != 0:
        return None
    wl = oracle_sample(args.cpu_sample)
    prob = O.Problem.from_tensor(wl.u, wl.D, theta=3e-4, lam_mode="literal")
    g = O.init_equilibrium(wl.phi0, wl.u)
    for k in range(args.warmup):
        g = O.step(g, prob, k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        g = O.step(g, prob, args.warmup + k)
    dt = time.perf_counter() - t0
    N = int(np.prod(wl.dims))
    v = N * args.steps / dt / 1e6
    sample = f"{args.steps} steps of the bench physics on a {wl.dims[0]}^3 periodic box (FP64 oracle, torch CPU)"
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="f32", choices=["f16dev", "bf16dev", "f32"],
                    help="headline (chosen) form")
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--dims", type=int, nargs=3, default=None, metavar=("NX", "NY", "NZ"),
                    help="with --only: a box of this shape instead of the cube (smaller profiling cases)")
    ap.add_argument("--err-steps", type=int, default=200)
    ap.add_argument("--cpu-sample", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=100,
                    help="steps per mode of the 512-domain sweep (0 skips it)")
    ap.add_argument("--step-kernel", type=int, default=0, choices=[0, 1, 2, 3],
                    help="step implementation: 0 auto, 1 per-node gathers, 2 staged rows, 3 pipelined rows")
    ap.add_argument("--workload", default="plume", choices=["plume", "heterogeneous"],
                    help="with --only: time the 256^3 plume (default) or the 384^3 heterogeneous workload")
    ap.add_argument("--only", default=None, choices=["f16dev", "bf16dev", "f32", "f64"],
                    help="time one form only (profiling runs)")
    ap.add_argument("--late-start", type=int, default=1800, help="first step of the late window")
    ap.add_argument("--late-window", type=int, default=200, help="steps timed late in the run (0 skips)")
    ap.add_argument("--skip-extra", action="store_true",
                    help="skip the heterogeneous, adjoint and D2Q9 workloads")
    ap.add_argument("--het-size", type=int, default=384)
    ap.add_argument("--het-steps", type=int, default=100)
    ap.add_argument("--het-err-steps", type=int, default=20)
    ap.add_argument("--adj-size", type=int, default=64)
    ap.add_argument("--adj-steps", type=int, default=500)
    ap.add_argument("--d2-size", type=int, default=4096)
    ap.add_argument("--d2-steps", type=int, default=200)
    ap.add_argument("--d2-err-steps", type=int, default=100)
    ap.add_argument("--d2-only", default=None, choices=["f64", "f32"],
                    help="time one D2Q9 form alone on the field workload and print its block")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        # the oracle runs on the host cores of rank 0 only; other ranks exit without work
        rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
        line = run_reference(args, rank, world, None)
        if rank == 0 and line is not None:
            print(json.dumps(line), flush=True)
        return
    rank, world, local, dist = dist_setup(args.gpus)
    line = run_ours(args, rank, world, local, dist)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
