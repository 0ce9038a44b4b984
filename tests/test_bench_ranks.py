"""bench.py's multi-rank host logic on CPU (gloo, world size 2): every rank of
`bench.py --gpus N` factors its own replica (the path has no data-path
collective), the job's time is the slowest rank's, and the reported value is
the whole job's throughput.  The reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(times[rank], dist)
        out.put((rank, slowest, bench.job_rate(world, 1000.0, slowest)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_whole_job_rate():
    world, times = 2, [0.25, 0.75]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in got:
        assert slowest == max(times)            # every rank sees the slowest time
        assert rate == world * 1000.0 / 0.75     # both replicas' work over that time


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(1.5, None) == 1.5
    assert bench.job_rate(1, 10.0, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(None) is None   # rank 1 returns before any work
    assert buf.getvalue() == ""
