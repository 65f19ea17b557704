"""The N>1 path of bench.py on CPU: two gloo ranks run the replicated
workload (each rank its own copy, no data-path collective), rank 0 prints
one JSON line with the aggregate, the other rank prints nothing."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_two_gloo_ranks():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--config", "0"]
    out = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_max_over_ranks_and_barrier_with_gloo():
    code = r'''
import os, sys, torch, torch.distributed as dist
sys.path.insert(0, os.environ["ROOT"])
import bench
dist.init_process_group("gloo")
r = dist.get_rank()
bench.barrier(2)
m = bench.max_over_ranks(1.5 + r, 2)
with open(os.environ["OUT"] + "." + str(r), "w") as f:   # one file per rank: no interleaved stdout
    f.write(f"{r} {m}")
dist.destroy_process_group()
'''
    import tempfile
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "ranks.py")
        with open(path, "w") as f:
            f.write(code)
        env = dict(os.environ, CUDA_VISIBLE_DEVICES="", ROOT=ROOT, OUT=os.path.join(tmp, "result"))
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
               "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), path]
        out = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, env=env, timeout=300)
        assert out.returncode == 0, out.stderr[-2000:]
        res = sorted(open(os.path.join(tmp, f"result.{r}")).read().split() for r in range(2))
    assert res == [["0", "2.5"], ["1", "2.5"]]
