"""Sharding a batch of independent tanks over ranks (one process per GPU).

The tanks of a batch are independent pressure equations, so splitting them
needs no collective on the data path: ``partition_tanks`` (the C ABI's
gfm_partition_tanks, host only) gives every rank the same tank -> rank table
from the tanks' cell counts, each rank solves its own tanks in one batched
launch, and ``gather_tank_records`` collects the small per-tank records
(solve info, timings) on every rank afterwards.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import GFM_OK, GFMError, load_library

__all__ = ["partition_tanks", "tanks_of_rank", "gather_tank_records"]


def partition_tanks(cells, n_ranks: int):
    """Rank of each tank and the cells each rank gets (gfm_partition_tanks)."""
    c = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
    out = np.empty(c.size, dtype=np.int32)
    load = np.empty(int(n_ranks), dtype=np.int64)
    st = load_library().gfm_partition_tanks(c.ctypes.data_as(ct.c_void_p), int(c.size), int(n_ranks),
                                            out.ctypes.data_as(ct.c_void_p), load.ctypes.data_as(ct.c_void_p))
    if st != GFM_OK:
        raise GFMError(st, "gfm_partition_tanks: cells must be >= 1 and there must be at least one tank and rank")
    return out, load


def tanks_of_rank(rank_of_tank, rank: int) -> list:
    """The tanks one rank solves, in ascending tank order."""
    return [int(t) for t in np.nonzero(np.asarray(rank_of_tank) == rank)[0]]


def gather_tank_records(records: dict, world: int, group=None) -> dict:
    """Merge every rank's {tank: record} into one dict on every rank (one
    all_gather of small host objects after the solves; nothing on the data
    path).  A tank reported by two ranks is an error."""
    if world <= 1:
        return dict(records)
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, dict(records), group=group)
    out = {}
    for part in parts:
        for t, rec in part.items():
            if t in out:
                raise RuntimeError(f"tank {t} was solved by two ranks")
            out[t] = rec
    return out
