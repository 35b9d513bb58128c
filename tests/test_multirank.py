"""The N > 1 launch of bench.py (one replica per rank, weak scaling) on CPU
ranks over gloo: process-group set-up from the torchrun environment, the
max-over-ranks time, the whole-job rate, and a reference arm that only
rank 0 runs."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    os.environ["CUDA_VISIBLE_DEVICES"] = ""  # CPU ranks: gloo
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    r, local, w = bench._dist()
    assert dist.get_backend() == "gloo"
    ms = bench.max_over_ranks(10.0 + 5.0 * r, w, "cpu")
    rate = bench.job_rate(1000.0, w, ms)
    q.put((r, w, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms, rate in out:
        assert w == world
        assert ms == 15.0  # the slower rank's time, on every rank
        assert rate == pytest.approx(2 * 1000.0 / 15e-3)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload = "tank2d"
        gpus = 2
        steps = 1
        warmup = 0

    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(Args(), rank=1, world=2) is None
    assert buf.getvalue() == ""
