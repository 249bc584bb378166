"""The multi-process side of bench.py on CPU (gloo, world size 2): the
max-over-ranks timing and barrier, rank-dependent replicas, and the
reference arm under torchrun (rank 0 alone works and prints one line)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    m = bench.allmax(1.5 + rank, world)
    bench.barrier(world)
    dist.destroy_process_group()
    with open(out + f".{rank}", "w") as fh:
        fh.write(repr(m))


def test_allmax_and_barrier_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = free_port()
    out = str(tmp_path / "m")
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        assert float(open(out + f".{r}").read()) == 2.5


def test_replicas_differ_by_rank():
    sys.path.insert(0, ROOT)
    import bench
    a, b = bench.workload("slab-32", 0), bench.workload("slab-32", 1)
    assert a.mesh == b.mesh and a.n == b.n
    assert not np.array_equal(a.x, b.x)
    assert bench.workload("slab-32", 0).seed == a.seed


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0
