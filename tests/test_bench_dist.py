"""The multi-rank path of bench.py on CPU: gloo, world size 2.

bench.py runs one independent replica per rank (no data-path collective); the
only cross-rank step is gathering every rank's work and time to form the
whole-job throughput.  These tests run that gather on two CPU ranks and the
reference arm under torch.distributed.run.
"""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    work = [1000.0 * (rank + 1), 2.0 + rank]          # rank 0: 1000 in 2 s; rank 1: 2000 in 3 s
    gathered = bench.allgather_floats(work, world)
    value, tmax = bench.aggregate([g[0] for g in gathered], [g[1] for g in gathered])
    out.put((rank, value, tmax, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_throughput_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tmax, gathered in res:
        assert gathered == [[1000.0, 2.0], [2000.0, 3.0]]
        assert tmax == 3.0
        assert value == pytest.approx(3000.0 / 3.0)


def test_aggregate_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate([5.0], [2.0]) == (2.5, 2.0)
    assert bench.allgather_floats([1.0, 2.0], 1) == [[1.0, 2.0]]


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1", "--particles", "2048"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["unit"] == "particle-steps/s"
    assert rec["value"] > 0 and rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0
