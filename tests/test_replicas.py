"""Multi-rank path on CPU (gloo, world size 2): sharding covers every unit once, and the
merged violation log of two shards equals the log of the whole stream (oracle)."""
import os
import tempfile

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import agile_synth as syn
import oracle
from paper_2606_06697_b300.abi import ViolationRecord
from paper_2606_06697_b300.replicas import allreduce_record, merge_records, shard


def to_record(log, client=0):
    return ViolationRecord(log.key, log.addr, log.width, log.verdict, log.site, log.range_id,
                           client, 0, log.count)


def test_shard_covers_everything():
    for n in (0, 1, 7, 100, 12345):
        for w in (1, 2, 3, 8):
            parts = [shard(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(w - 1))


def _worker(rank, world, init, q):
    dist.init_process_group("gloo", init_method=init, rank=rank, world_size=world)
    t = syn.batch_table()
    addr, width, _ = syn.batch_accesses(t, 50_000)
    lo, hi = shard(len(addr), rank, world)
    _, _, log = oracle.check_batch(t, addr[lo:hi], width[lo:hi], method="sorted")
    # shard-local keys are indices within the shard: make them global
    rec = to_record(log)
    if rec.count:
        rec = ViolationRecord(rec.key + lo, *list(rec.__dict__.values())[1:])
    merged = allreduce_record(rec)
    q.put((rank, merged))
    dist.destroy_process_group()


def test_two_rank_merge_equals_whole():
    t = syn.batch_table()
    addr, width, _ = syn.batch_accesses(t, 50_000)
    _, _, whole = oracle.check_batch(t, addr, width, method="sorted")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with tempfile.TemporaryDirectory() as d:
        init = "file://" + os.path.join(d, "rdv")
        procs = [ctx.Process(target=_worker, args=(r, 2, init, q)) for r in range(2)]
        for p in procs:
            p.start()
        res = [q.get(timeout=120) for _ in range(2)]
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
    for _, merged in res:
        assert (merged.key, merged.addr, merged.width, merged.verdict, merged.range_id,
                merged.count) == (whole.key, whole.addr, whole.width, whole.verdict,
                                  whole.range_id, whole.count)


def test_merge_records_empty_and_status():
    a = ViolationRecord(0, 0, 0, 0, 0, 0xFFFFFFFF, 1, 0, 0)
    b = ViolationRecord(0, 0, 0, 0, 0, 0xFFFFFFFF, 1, 1, 0)
    m = merge_records([a, b])
    assert m.count == 0 and m.status == 1
    c = ViolationRecord(5, 50, 4, 1, 2, 7, 1, 0, 3)
    d = ViolationRecord(5, 50, 4, 1, 1, 7, 1, 0, 2)
    m = merge_records([c, d, a])
    assert m.site == 1 and m.count == 5
