"""The multi-process path of bench.py on the CPU: two `gloo` ranks over
127.0.0.1 take the maximum of their timings (the job's time is the slowest
replica's) and report the whole job's rate; the reference arm does its work
on rank 0 only.  The path has no data-path collective (independent replicas),
so these host-side steps are all there is to cover without GPUs."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local = [10.0 + 2.0 * rank, 3.0 - rank]  # ms of this replica: step time and another timing
    got = bench.max_over_ranks(dist, local, "cpu")
    dist.barrier()
    rate = bench.whole_job_rate(world, 393216 * 100, got[0])
    q.put((rank, got, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == [12.0, 3.0]
        assert rate == pytest.approx(2 * 393216 * 100 / 12e-3)


def test_single_process_reduction_is_identity():
    import bench
    assert bench.max_over_ranks(None, [1.5, 2.5], "cpu") == [1.5, 2.5]
    assert bench.whole_job_rate(1, 1000, 2.0) == pytest.approx(5e5)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun every rank runs bench.py; a reference line comes from
    rank 0 alone, the other ranks exit 0 without work or output."""
    import bench

    class A:
        impl = "reference"
        workload = "plate"
        gpus = 2
        steps = 1
        warmup = 3
        seed = 0
        ref_seconds = 10.0

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(A(), 2, 1) == 0
    assert buf.getvalue() == ""
