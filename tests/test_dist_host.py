"""The N > 1 path on CPU: replicas only, so the one cross-rank step is the
benchmark's max-over-ranks timing (gloo, world size 2), and under torchrun the
reference arm runs on rank 0 alone while the other ranks exit without work."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, values, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    out[rank] = bench.max_over_ranks(values[rank], ws, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world_size_2():
    ws, port = 2, _free_port()
    values = [12.5, 31.25]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, port, values, out), nprocs=ws, join=True)
        assert dict(out) == {0: 31.25, 1: 31.25}


def test_max_over_ranks_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(7.0, 1, torch.device("cpu")) == 7.0


def test_reference_arm_under_torchrun_prints_once_on_rank_0():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--ref-budget", "2"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
