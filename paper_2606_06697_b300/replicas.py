"""Replicas across GPUs: the guard's checks are independent, so a sharded run exchanges
nothing while it works. At the end each rank holds its own violation log; the job's
log is the record with the smallest (key, site, verdict, width, range) over the ranks and
the sum of their counts -- the same minimum the device log keeps. Host-side, through
torch.distributed (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

from dataclasses import astuple

import torch.distributed as dist

from .abi import ViolationRecord


def _order(r: ViolationRecord):
    return (r.key, r.site, r.verdict, r.width, r.range_id)


def merge_records(records):
    """Combine per-shard records: smallest key wins, counts add, status bits or."""
    live = [r for r in records if r.count]
    total = sum(r.count for r in records)
    status = 0
    for r in records:
        status |= r.status
    if not live:
        base = records[0]
        return ViolationRecord(0, 0, 0, 0, 0, base.range_id, base.client, status, 0)
    best = min(live, key=_order)
    return ViolationRecord(best.key, best.addr, best.width, best.verdict, best.site,
                           best.range_id, best.client, status, total)


def allreduce_record(rec: ViolationRecord, group=None) -> ViolationRecord:
    """Every rank gets the merged record of all ranks."""
    gathered = [None] * dist.get_world_size(group)
    dist.all_gather_object(gathered, astuple(rec), group=group)
    return merge_records([ViolationRecord(*t) for t in gathered])


def shard(n: int, rank: int, world: int):
    """Contiguous [lo, hi) of n units for this rank (the first n % world ranks get one more)."""
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)
