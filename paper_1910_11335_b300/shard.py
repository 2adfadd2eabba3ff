"""Multi-GPU sharding of independent source positions (one process per GPU).

The CT projections of the batching form are independent solves: one set of
source positions is partitioned over the ranks (rank r takes positions r,
r + R, r + 2R, ... of the set), every rank holds its own replica of the
phantom and the cross sections, and the ranks' results are gathered to rank 0
on the host. Nothing is exchanged on the device data path: a single solve does
not shard (groups are sequential and the directions of one iteration share
their moments), so there is no collective to overlap.

Host logic only; the solves themselves are the library's (or, in the CPU
tests, the oracle's).
"""
from __future__ import annotations

from typing import Dict, List, Optional


def partition(n_sources: int, world: int, rank: int) -> List[int]:
    """Indices into one source set of n_sources positions that rank `rank` of
    `world` solves: rank, rank + world, ... (strided, so that every rank's
    share spreads around the ring)."""
    if world < 1 or not 0 <= rank < world or n_sources < 0:
        raise ValueError(f"bad partition request: {n_sources} sources, rank {rank} of {world}")
    return list(range(rank, n_sources, world))


def gather_to_root(local: Dict[int, object], world: int, rank: int) -> Optional[List[object]]:
    """Gather every rank's {global source index: result} to rank 0 on the host
    (torch.distributed.gather_object on the default process group) and return
    rank 0 the results ordered by global source index; other ranks get None.
    Raises if two ranks report the same source or a source is missing."""
    if world == 1:
        parts = [local]
    else:
        import torch.distributed as dist
        parts = [None] * world if rank == 0 else None
        dist.gather_object(local, parts, dst=0)
    if rank != 0:
        return None
    merged: Dict[int, object] = {}
    for part in parts:
        for k, v in part.items():
            if k in merged:
                raise ValueError(f"source {k} reported by two ranks")
            merged[k] = v
    keys = sorted(merged)
    if keys != list(range(len(keys))):
        raise ValueError(f"gathered sources are not 0..{len(keys) - 1}: {keys[:8]}...")
    return [merged[k] for k in keys]
