"""Sharding a batch of tanks across ranks (no data-path collective): the
partition table of gfm_partition_tanks (host C ABI, no GPU), and the
gathered per-tank records of two gloo ranks on CPU, each rank solving its
own tanks (here with the CPU oracle, which stands in for the GPU batch: the
test is about which rank solves what and what gets gathered)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SMALL = dict(ntanks=10, seed0=4100, nx_range=(12, 40), ny_range=(6, 20))


def _cells(**kw):
    return [nx * ny for nx, ny, _, _ in cases.batch_shapes(**kw)]


def _shard():
    from paper_1804_01130_gb300 import shard
    return shard


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_every_tank_lands_on_exactly_one_rank_within_the_bound(world):
    shard = _shard()
    cells = np.array(_cells())  # the 64-tank workload's sizes
    rank_of, load = shard.partition_tanks(cells, world)
    assert rank_of.shape == (64,) and rank_of.min() >= 0 and rank_of.max() < world
    per_rank = [shard.tanks_of_rank(rank_of, r) for r in range(world)]
    assert sorted(t for ts in per_rank for t in ts) == list(range(64))
    for r in range(world):
        assert load[r] == cells[per_rank[r]].sum()
    # list-scheduling bound on the busiest rank
    assert load.max() <= cells.sum() / world + (1 - 1 / world) * cells.max()
    # and the longest-first order keeps 64 tanks within 1% of the ideal on 2 ranks
    if world == 2:
        assert load.max() <= 1.01 * cells.sum() / 2
    # a pure function of the counts
    again, _ = shard.partition_tanks(cells, world)
    assert np.array_equal(again, rank_of)


def test_partition_rejects_bad_arguments():
    shard = _shard()
    import paper_1804_01130_gb300 as g
    with pytest.raises(g.GFMError):
        shard.partition_tanks([10, 0, 5], 2)
    with pytest.raises(g.GFMError):
        shard.partition_tanks([10, 5], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _solve_tanks(only):
    import oracle
    oracle.set_threads(1)  # the same summation order in every process
    out = {}
    for t, c in zip(only, cases.batch_cases(**SMALL, only=only)):
        p, _, _, info = oracle.solve(c, rtol=1e-10, direct=False)
        out[t] = {"iters": info["iters"], "status": info["status"], "n": c.n, "p_sum": float(np.sum(p)),
                  "p_norm": float(np.linalg.norm(p))}
    return out


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    os.environ["CUDA_VISIBLE_DEVICES"] = ""
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_1804_01130_gb300 import shard
    dist.init_process_group("gloo")
    rank_of, _ = shard.partition_tanks(_cells(**SMALL), world)
    mine = shard.tanks_of_rank(rank_of, rank)
    local = _solve_tanks(mine)
    merged = shard.gather_tank_records(local, world)
    q.put((rank, mine, merged))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_single_rank_records():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    owned = sorted(t for _, mine, _ in out for t in mine)
    assert owned == list(range(SMALL["ntanks"]))  # each tank solved exactly once
    single = _solve_tanks(list(range(SMALL["ntanks"])))
    for _, _, merged in out:
        assert merged == single  # every rank ends with every tank's record, as one rank would


def test_gather_refuses_a_tank_solved_twice(monkeypatch):
    shard = _shard()
    import torch.distributed as dist

    def fake_all_gather_object(parts, obj, group=None):
        parts[0] = {3: {"iters": 1}}
        parts[1] = {3: {"iters": 1}}

    monkeypatch.setattr(dist, "all_gather_object", fake_all_gather_object)
    with pytest.raises(RuntimeError, match="two ranks"):
        shard.gather_tank_records({3: {"iters": 1}}, 2)
