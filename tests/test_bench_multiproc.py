"""bench.py under torchrun with two ranks on the CPU (gloo): the host-side
logic of the replica path -- the process group, the barrier and the
max-over-ranks timing -- and the reference arm, where rank 0 alone runs and
prints one JSON line and the other rank exits 0 without work."""
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


WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import bench
rank, world, local = bench._dist()
bench._barrier(world)
m = bench._max_over_ranks(10.0 + rank, world, "cpu")
sys.stdout.write(f"RESULT {{rank}} {{world}} {{m}}\n")   # one write: ranks share the pipe
sys.stdout.flush()
"""


def test_max_over_ranks_and_barrier_with_gloo(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT))
    env = dict(os.environ, FV_BENCH_BACKEND="gloo")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node=2", "--master-addr", "127.0.0.1", "--master-port",
                        str(_free_port()), str(script)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l.split() for l in r.stdout.splitlines() if l.startswith("RESULT")]
    assert sorted(int(l[1]) for l in lines) == [0, 1]
    assert all(int(l[2]) == 2 and float(l[3]) == 11.0 for l in lines)


def test_reference_arm_two_ranks_prints_one_line():
    env = dict(os.environ, FV_BENCH_BACKEND="gloo")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node=2", "--master-addr", "127.0.0.1", "--master-port",
                        str(_free_port()), os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "zone-updates/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
