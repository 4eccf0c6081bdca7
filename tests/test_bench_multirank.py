"""Host logic of bench.py's multi-rank path, on CPU with the gloo backend (world size 2):
max/sum over ranks and barriers, round-robin sharding of independent domains, and the
reference arm under torchrun (rank 0 alone prints one JSON line)."""
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_partitions_units():
    sys.path.insert(0, ROOT)
    import bench
    items = list(range(37))
    parts = [bench.shard(items, r, 4) for r in range(4)]
    assert sorted(x for p in parts for x in p) == items
    assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1


WORKER = r"""
import os, sys
sys.path.insert(0, os.environ["ROOT"])
import bench
rank, world, local, dist = bench.dist_setup(2)
assert world == 2 and dist is not None
v = bench.max_over_ranks(float(rank + 1) * 1.5, dist)
s = bench.sum_over_ranks(float(rank + 1), dist)
bench.barrier(dist)
print(f"RANK{rank} max={v} sum={s}", flush=True)
dist.destroy_process_group()
"""


def _torchrun(args, env_extra=None, timeout=240):
    env = dict(os.environ, ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
    if env_extra:
        env.update(env_extra)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(29500 + os.getpid() % 1000)] + args
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_gloo_reductions_two_ranks(tmp_path):
    w = tmp_path / "worker.py"
    w.write_text(WORKER)
    r = _torchrun([str(w)])
    assert r.returncode == 0, r.stderr[-2000:]
    # both ranks share stdout, so their lines may interleave: match the records, not the lines
    lines = sorted(re.findall(r"RANK\d max=[0-9.]+ sum=[0-9.]+", r.stdout))
    assert lines == ["RANK0 max=3.0 sum=3.0", "RANK1 max=3.0 sum=3.0"], r.stdout


def test_reference_arm_two_ranks_prints_one_line():
    r = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "3", "--warmup", "3",
                   "--cpu-sample", "10"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
