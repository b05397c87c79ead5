"""Many clients in one persistent guarded launch: every client's output and log equal
its own single launch and the oracle; graph replays equal eager launches; the
autotuner returns a working configuration and reuses its cache."""
import os
import tempfile

import numpy as np
import pytest
import torch

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag
from paper_2606_06697_b300.clients import ClientSet

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def small_specs(n=24, seed=syn.SEED_BASE + 40):
    return syn.client_specs(n, seed=seed, median=48 * 1024, lo=4 * 1024, hi=512 * 1024,
                            table_lo=8, table_hi=300)


def same(a, b):
    (oa, la), (ob, lb) = a, b
    assert oa.view(np.uint32).tobytes() == ob.view(np.uint32).tobytes()
    assert (la.count, la.key, la.addr, la.width, la.verdict, la.site, la.range_id, la.client) == \
        (lb.count, lb.key, lb.addr, lb.width, lb.verdict, lb.site, lb.range_id, lb.client)


def oracle_outputs(cs, which=None):
    """The oracle's output and log for every client (or the clients `which`), from the
    device inputs."""
    res = []
    host = cs.arena.cpu().numpy()
    for i, c in enumerate(cs.clients):
        if which is not None and i not in which:
            continue
        s, n, b = c["spec"], c["n"], c["buf"]
        off, span = c["arena_off"], c["span"]
        if s["op"] == "copy":
            bv = cs.view(c, "b", torch.float32, n).cpu().numpy()
            out, log = oracle.stream("copy", c["ranges"], {"a": b["a"], "b": b["b"]}, bv, None,
                                     np.zeros(n, np.float32), 3.0, cs.policy)
        else:
            arena = host[off:off + span].copy()
            if s["op"] == "gather":
                arena[b["out"] - cs.base - off:b["out"] - cs.base - off + 4 * n] = 0
                va = {"idx": b["idx"], "t": b["t"], "out": b["out"]}
            else:
                arena[b["bins"] - cs.base - off:b["bins"] - cs.base - off + 4 * syn.HIST_BINS] = 0
                va = {"idx": b["idx"], "t": b["bins"]}
            log = oracle.irregular(s["op"], c["ranges"], arena, cs.base + off, va, n, cs.policy)
            if s["op"] == "gather":
                o = b["out"] - cs.base - off
                out = arena[o:o + 4 * n].view(np.float32)
            else:
                o = b["bins"] - cs.base - off
                out = arena[o:o + 4 * syn.HIST_BINS].view(np.int32)
        res.append((out, log))
    return res


@pytest.mark.parametrize("policy", ["poison", "report"])
def test_batch_equals_single_and_oracle(policy):
    cs = ClientSet(small_specs(), DEV, log2_pages=(16, 21), frac_bad=0.01, policy=policy)
    n = len(cs.clients)
    buf = torch.empty(ag.agile_batch_device_bytes(n), dtype=torch.uint8, device=DEV)
    for i in range(n):
        cs.run_single(i, 1)
    single = cs.outputs()
    want = oracle_outputs(cs)
    for got, exp in zip(single, want):
        (o, rec), (eo, elog) = got, exp
        assert o.view(np.uint32).tobytes() == eo.view(np.uint32).tobytes()
        assert (rec.count, rec.key, rec.addr, rec.width, rec.verdict, rec.site, rec.range_id) == \
            (elog.count, elog.key, elog.addr, elog.width, elog.verdict, elog.site, elog.range_id)
    assert any(r.count for _, r in single)
    for variant in (0, 1):
        for tile, spans, bps in ((512, True, 2), (4096, False, 1), (65536, True, 1)):
            cs.reset()
            ag.agile_batch_upload(cs.work(variant), tile, buf)
            ag.agile_batch_launch(buf, n, tile, spans, bps)
            for a, b in zip(cs.outputs(), single):
                same(a, b)


def test_batch_graph_replay_and_relist():
    cs = ClientSet(small_specs(16, seed=syn.SEED_BASE + 41), DEV, log2_pages=(21,))
    n = len(cs.clients)
    buf = torch.empty(ag.agile_batch_device_bytes(n), dtype=torch.uint8, device=DEV)
    ag.agile_batch_upload(cs.work(0), 4096, buf)
    ag.agile_batch_launch(buf, n, 4096)
    eager = cs.outputs()
    g = ag.agile_batch_graph_create(buf, n, 4096)
    for _ in range(3):
        cs.reset()
        g.launch()
        torch.cuda.synchronize()
        for a, b in zip(cs.outputs(), eager):
            same(a, b)
    # a new work list of the same length: the unguarded twins, then back
    cs.reset()
    ag.agile_batch_upload(cs.work(0, guarded=False), 4096, buf)
    g.launch()
    torch.cuda.synchronize()
    for (o, _), (eo, _) in zip(cs.outputs(), eager):
        assert o.tobytes() == eo.tobytes()
    g.destroy()


def test_autotune_and_cache():
    cs = ClientSet(small_specs(12, seed=syn.SEED_BASE + 42), DEV, log2_pages=(16, 21))
    n = len(cs.clients)
    buf = torch.empty(ag.agile_batch_device_bytes(n), dtype=torch.uint8, device=DEV)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        best = ag.agile_batch_autotune([cs.work(0), cs.work(1)], [512, 4096], buf, reps=2,
                                       cache_path=path)
        assert best["tile"] in (512, 4096) and best["variant"] in (0, 1) and not best["cached"]
        again = ag.agile_batch_autotune([cs.work(0), cs.work(1)], [512, 4096], buf, reps=2,
                                        cache_path=path)
        assert again["cached"] and again["tile"] == best["tile"]
    cs.reset()
    ag.agile_batch_upload(cs.work(best["variant"]), best["tile"], buf)
    ag.agile_batch_launch(buf, n, best["tile"], best["span_checks"], best["blocks_per_sm"])
    tuned = cs.outputs()
    cs.reset()
    for i in range(n):
        cs.run_single(i, 0)
    for a, b in zip(tuned, cs.outputs()):
        same(a, b)


def test_batch_rejects_bad_items():
    x = torch.zeros(64, dtype=torch.float32, device=DEV)
    buf = torch.empty(ag.agile_batch_device_bytes(1), dtype=torch.uint8, device=DEV)
    bad = ag.make_work("copy", None, x.data_ptr() + 4, x, None, 8)
    with pytest.raises(ag.AgileError) as e:
        ag.agile_batch_upload([bad], 512, buf)
    assert e.value.code == -12
    with pytest.raises(ag.AgileError):
        ag.agile_batch_upload([ag.make_work("copy", None, x, x, None, 8)], 100, buf)
