"""The multi-rank (N > 1) logic of bench.py on the CPU, with gloo ranks on
127.0.0.1: every rank times its own fits (weak scaling, no data-path
exchange), the job's time is the slowest rank's, the rate counts the units
of all ranks, and only rank 0 prints."""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = bench._env_rank()
    local_ms = 10.0 + 7.5 * rank                  # rank 1 is the slow one
    slowest = bench.max_over_ranks(local_ms)
    rate = bench.whole_job_rate(30, w, slowest)
    dist.destroy_process_group()
    out.put((rank, r, lr, w, slowest, rate))


def test_two_gloo_ranks_report_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, lr, w, slowest, rate in got:
        assert (r, lr, w) == (rank, rank, 2)
        assert slowest == 17.5                    # both ranks agree on the slowest time
        assert rate == pytest.approx(2 * 30 / 0.0175)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(10, 1, 500.0) == pytest.approx(20.0)


def test_reference_arm_prints_once_under_torchrun():
    """`bench.py --impl reference` launched as two ranks: rank 0 times the
    oracle and prints one line, rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
