"""The committed per-launch DRAM traffic (profiles/step_traffic.txt) that bench.py reports as
`roofline.traffic`: it must have been taken on the kernel sources in the tree (bench.py reports
null otherwise), it must cover every storage form the bench times, and each figure must sit near
the form's algorithmic bytes per launch on the 256^3 plume (traffic far above them would mean
re-reads; far below, a kernel that does not do the work)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    return bench


def _entries():
    vals = {}
    for line in open(os.path.join(ROOT, "profiles", "step_traffic.txt")):
        parts = line.split()
        if len(parts) == 2 and not line.startswith("#"):
            vals[parts[0]] = parts[1]
    return vals


def test_traffic_taken_on_current_kernels():
    bench = _bench()
    assert _entries()["kernel_hash"] == bench.kernel_hash()
    for form in ("f32", "f16dev", "bf16dev", "f64"):
        assert bench.ncu_traffic(form) is not None, form


def test_traffic_near_algorithmic_bytes():
    bench = _bench()
    nodes = 256 ** 3
    for form in ("f32", "f16dev", "bf16dev", "f64"):
        algorithmic = bench.BYTES_PER_NODE[form] * nodes
        ratio = bench.ncu_traffic(form) / algorithmic
        assert 0.9 < ratio < 1.1, (form, ratio)
