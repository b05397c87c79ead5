"""The serving worker: validation rejects every bad pointer with the oracle's verdict,
continuous batching gives the same results as serving one request at a time, admission
never exceeds the memory budget."""
import numpy as np
import pytest
import torch

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag
from paper_2606_06697_b300.serving import ServedClients, latency_stats, serve

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
VERDICT = {"protected": 1, "freed": 4, "straddle": 3}


def small():
    specs = syn.serve_specs(12, seed=syn.SEED_BASE + 60, median=96 * 1024, lo=64 * 1024,
                            hi=1 << 20)
    return ServedClients(specs, DEV)


def snapshot(cs):
    return [cs.output(i, k).cpu().numpy().tobytes() for i in range(len(cs.specs))
            for k in range(syn.SERVE_SLOTS)]


def test_validation_matches_oracle_and_rejects_all_bad():
    cs = small()
    gen = syn.serve_requests(cs.layouts, 20000, 600, frac_bad=0.03)
    done, _ = serve(cs, gen)
    assert len(done) == len(gen)
    by_tag = {c.tag: c for c in done}
    for k, g in enumerate(gen):
        c = by_tag[k]
        r, freed, span, off, sizes, n = cs.layouts[g["client"]]
        live = ~freed
        rr = r.shifted(cs.base + cs.off[g["client"]])
        t = syn._ranges(rr.base[live], rr.size[live], rr.kind[live], rr.ident[live])
        ptr = np.array([cs.addr(g["client"], o) for o, _ in g["args"]], np.uint64)
        nb = np.array([b for _, b in g["args"]], np.uint64)
        ov, _ = oracle.validate(t, ptr, nb)
        if g["bad"] is None:
            assert c.status == 0 and (ov == 0).all()
        else:
            first = int(np.flatnonzero(ov != 0)[0])
            assert c.status == 1 and c.bad_arg == first and c.verdict == ov[first]
            assert c.verdict == VERDICT[g["bad"]]
    assert sum(g["bad"] is not None for g in gen) == sum(c.status == 1 for c in done)


def test_continuous_batching_equals_one_at_a_time():
    cs = small()
    gen = syn.serve_requests(cs.layouts, 50000, 800, frac_bad=0.0)
    mixed, _ = serve(cs, gen, continuous=True, max_batch=32, max_inflight=4)
    st = latency_stats(gen, mixed)
    assert st["served"] == len(gen) and st["launches"] < len(gen)   # requests shared launches
    for c in mixed:                      # the completion's times follow the request's path
        assert c.arrival_ns <= c.seen_ns <= c.admit_ns <= c.queued_ns <= c.done_ns
    got = snapshot(cs)
    logs = [ag.agile_violation_log_read(cs.log(i))[1].count for i in range(len(cs.specs))]
    cs.reset()
    alone, _ = serve(cs, gen, continuous=False)
    assert latency_stats(gen, alone)["launches"] == len(gen)
    assert snapshot(cs) == got
    assert logs == [0] * len(cs.specs)


def test_admission_respects_budget():
    cs = small()
    gen = syn.serve_requests(cs.layouts, 100000, 300, frac_bad=0.0)
    reqs = [cs.request(k, g) for k, g in enumerate(gen)]
    biggest = max(r.mem_bytes for r in reqs)
    budget = 2 * biggest
    done, peak = serve(cs, gen, budget=budget)
    assert all(c.status == 0 for c in done) and len(done) == len(gen)
    assert 0 < peak <= budget
    done, _ = serve(cs, gen[:5], budget=biggest // 4)
    assert any(c.status == -11 for c in done)            # a request that can never fit
