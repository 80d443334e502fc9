"""Replica runs (one process per GPU, no data-path collective): the job time
is the slowest rank's and the work is summed over ranks.  Checked with two
gloo ranks on the CPU; the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch, torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
r = dist.get_rank()
secs = [1.5, 2.0][r]
dofs = [100.0, 250.0][r]
t = bench.over_ranks(dist, torch, secs, "max", device="cpu")
n = bench.over_ranks(dist, torch, dofs, "sum", device="cpu")
print(f"RANK{r} {t} {n}", flush=True)
dist.destroy_process_group()
"""


def test_replica_aggregation_two_gloo_ranks(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    for r, (o, _) in enumerate(outs):
        line = [l for l in o.splitlines() if l.startswith(f"RANK{r}")][0]
        _, t, n = line.split()
        assert float(t) == 2.0 and float(n) == 350.0


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.over_ranks(None, None, 3.5, "max") == 3.5


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0 and out.stdout.strip() == ""
