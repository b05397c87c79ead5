"""Parity at the benchmark's full sizes, in the launch configurations it times: outputs
the oracle can compute one by one are compared with it, the rest through properties that
hold at any size (guarded equals unguarded on allowed accesses, denied accesses leave
memory untouched, histograms equal a count of the allowed keys)."""
import numpy as np
import pytest
import torch

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag
from gpu_util import DEV, device_table, new_log

pytestmark = pytest.mark.gpu


def _irregular_full(dist):
    n = 1 << 28
    r, span, off = syn.irregular_layout(n)
    idx, key, bad = syn.irregular_indices(n, dist=dist)
    arena = torch.empty(span, dtype=torch.uint8, device=DEV)
    base = arena.data_ptr()
    return n, r, off, idx, key, bad, arena, base


def _first_fault(rec, table, a, site=2):
    """Every field of the log's first record against the oracle's verdict for the access
    with the smallest address among the denied ones (4-byte element accesses)."""
    ov, orid, _ = oracle.check_batch(table, np.array([a], np.uint64), np.array([4], np.uint8),
                                     method="sorted")
    assert (rec.key, rec.addr, rec.width, rec.site, rec.verdict, rec.range_id) == \
        (a, a, 4, site, int(ov[0]), int(orid[0])), rec


def test_irregular_full_size_scatter_and_histogram():
    """Scatter: the guarded result equals an unguarded scatter of the allowed indices alone
    over the whole 16 GiB table region, protected tails included. Histogram: the guarded
    bins equal the count of the allowed keys, and the protected tail after them stays 0."""
    n, r, off, idx, key, bad, arena, base = _irregular_full("uniform")
    tbytes = off["bins"]
    tview = arena[:tbytes].view(torch.float32)
    g = torch.Generator(device=DEV).manual_seed(17)
    tview.uniform_(1, 2, generator=g)
    init = tview.clone()
    d_idx = arena[off["idx"]:off["idx"] + 8 * n].view(torch.int64)
    d_idx.copy_(torch.from_numpy(idx))
    d_bad = torch.from_numpy(bad).to(DEV)
    _, dev = device_table(r.shifted(base), 16)
    log = new_log()
    ag.agile_irregular_launch("scatter", dev, d_idx, base, None, n, "poison", log)
    rc, rec = ag.agile_violation_log_read(log)
    nb = int(bad.sum())
    assert rc == 1 and rec.count == nb and rec.site == 2 and rec.verdict == 1
    _first_fault(rec, r.shifted(base), base + 4 * int(idx[bad].min()))
    guarded = tview.clone()
    tview.copy_(init)
    good = d_idx[~d_bad].contiguous()
    ag.agile_irregular_launch("scatter", None, good, base, None, good.numel())
    assert torch.equal(guarded.view(torch.int32), tview.view(torch.int32))
    del guarded, init, good
    # histogram over the 2^20 bins
    bins = arena[off["bins"]:off["bins"] + 4 * (1 << 20) + 64 * 1024].view(torch.int32)
    bins.zero_()
    d_idx.copy_(torch.from_numpy(key))
    log = new_log()
    ag.agile_irregular_launch("hist", dev, d_idx, base + off["bins"], None, n, "poison", log)
    rc, rec = ag.agile_violation_log_read(log)
    assert rc == 1 and rec.count == nb
    _first_fault(rec, r.shifted(base), base + off["bins"] + 4 * int(key[bad].min()))
    want = torch.bincount(d_idx[~d_bad], minlength=1 << 20).to(torch.int32)
    assert torch.equal(bins[:1 << 20], want) and int(bins[1 << 20:].abs().sum()) == 0


def test_irregular_full_size_gather_zipf():
    """Zipf(1.1) gather: guarded equals unguarded except at the denied positions, which
    read 0; sampled outputs equal the table values the oracle's index rule names."""
    n, r, off, idx, key, bad, arena, base = _irregular_full("zipf")
    tview = arena[:off["bins"]].view(torch.float32)
    tview.uniform_(1, 2, generator=torch.Generator(device=DEV).manual_seed(18))
    d_idx = arena[off["idx"]:off["idx"] + 8 * n].view(torch.int64)
    d_idx.copy_(torch.from_numpy(idx))
    out = arena[off["out"]:off["out"] + 4 * n].view(torch.float32)
    _, dev = device_table(r.shifted(base), 21)
    log = new_log()
    ag.agile_irregular_launch("gather", dev, d_idx, base, out, n, "poison", log)
    rc, rec = ag.agile_violation_log_read(log)
    g = out.clone()
    ag.agile_irregular_launch("gather", None, d_idx, base, out, n)
    d_bad = torch.from_numpy(bad).to(DEV)
    assert torch.equal(g[~d_bad], out[~d_bad]) and bool((g[d_bad] == 0).all())
    assert rc == 1 and rec.count == int(bad.sum())
    _first_fault(rec, r.shifted(base), base + 4 * int(idx[bad].min()))
    sample = syn.Stream(19, 19).below(n, 2048)
    s_idx = torch.from_numpy(idx[sample]).to(DEV)
    assert torch.equal(g[torch.from_numpy(sample).to(DEV)],
                       torch.where(torch.from_numpy(bad[sample]).to(DEV), 0.0, tview[s_idx]))


def test_clients_full_size():
    """The benchmark's 256 clients (lognormal buffers, median 2 MiB; tables of 8-4096
    ranges), 0.1% of gather/histogram indices aimed at protected decoys: the CUDA-graph
    replay of the persistent launch at the tuned tile equals every client's own launch,
    and a sample of clients equals the oracle."""
    from paper_2606_06697_b300.clients import ClientSet
    from test_gpu_batch_clients import oracle_outputs, same
    cs = ClientSet(syn.client_specs(256), DEV, log2_pages=(16, 21), frac_bad=0.001)
    n = len(cs.clients)
    for i in range(n):
        cs.run_single(i, 0)
    single = cs.outputs()
    assert sum(1 for _, r in single if r.count) > 10
    buf = torch.empty(ag.agile_batch_device_bytes(n), dtype=torch.uint8, device=DEV)
    for variant, tile in ((0, 65536), (1, 16384)):
        cs.reset()
        ag.agile_batch_upload(cs.work(variant), tile, buf)
        gr = ag.agile_batch_graph_create(buf, n, tile, True, 2)
        gr.launch()
        torch.cuda.synchronize()
        for a, b in zip(cs.outputs(), single):
            same(a, b)
        gr.destroy()
    small = [i for i, c in enumerate(cs.clients) if c["n"] <= 1 << 20]
    pick = [small[j] for j in syn.Stream(20, 20).below(len(small), 8).tolist()]
    want = oracle_outputs(cs, set(pick))
    for i, (eo, elog) in zip(sorted(set(pick)), want):
        o, rec = single[i]
        assert o.view(np.uint32).tobytes() == eo.view(np.uint32).tobytes()
        assert (rec.count, rec.key, rec.addr, rec.width, rec.verdict, rec.site, rec.range_id) == \
            (elog.count, elog.key, elog.addr, elog.width, elog.verdict, elog.site, elog.range_id)
