"""Bounded violation list (Sec. V-E: report counts or logs would-be violations). Every
violation a kernel records in a log that has a list attached is also appended to the
list, until the list is full; later ones are only counted. The entries come in the order
the GPU took their slots, so they are compared with the oracle as a multiset -- all of
them when the list holds every violation, and as a sub-multiset, with the count of all
violations seen, when it overflows."""
import ctypes
from collections import Counter

import numpy as np
import pytest
import torch

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag
from gpu_util import DEV, assert_log_equal, device_table, new_log, to_dev
from test_gpu_ptx import EXITS
from test_gpu_stream import _fill, _hostile_layout

pytestmark = pytest.mark.gpu


def new_list(log, capacity):
    buf = torch.zeros(ag.list_bytes(capacity), dtype=torch.uint8, device=DEV)
    ag.agile_violation_list_attach(log, buf, capacity)
    return buf


def entries(recs):
    return Counter((r.key, r.addr, r.width, r.verdict, r.site, r.range_id) for r in recs)


def expected(addr, width, sites=None, key_is_index=True, r=None, verdicts=None, rids=None):
    """The oracle's multiset of records for the denied accesses among (addr, width)."""
    if verdicts is None:
        verdicts, rids, _ = oracle.check_batch(r, addr, width, method="sorted")
    sites = np.zeros(len(addr), np.uint32) if sites is None else sites
    d = np.flatnonzero(verdicts != 0)
    return Counter((int(i) if key_is_index else int(addr[i]), int(addr[i]), int(width[i]),
                    int(verdicts[i]), int(sites[i]), int(rids[i])) for i in d)


def check(recs, n_seen, exp, capacity):
    total = sum(exp.values())
    assert n_seen == total
    got = entries(recs)
    if total <= capacity:
        assert got == exp
    else:
        assert sum(got.values()) == capacity and not (got - exp)   # a sub-multiset
    for r in recs:
        assert r.count == 1 and r.status == 0


@pytest.mark.parametrize("capacity", [1 << 17, 1000])
def test_list_batch_check(capacity):
    """1M accesses of the batch workload: every denial, keyed by its index."""
    t = syn.batch_table()
    addr, width, _ = syn.batch_accesses(t, 1 << 20)
    _, dev = device_table(t, 21)
    d_addr, d_width = to_dev(addr.view(np.int64)), to_dev(width)
    d_v = torch.empty(len(addr), dtype=torch.uint8, device=DEV)
    log = new_log(client=6)
    lst = new_list(log, capacity)
    ag.agile_guard_check_batch(dev, d_addr, d_width, len(addr), d_v, log)
    rc, rec = ag.agile_violation_log_read(log)
    ov, orid, olog = oracle.check_batch(t, addr, width, method="sorted")
    assert (d_v.cpu().numpy() == ov).all()
    assert_log_equal(rec, olog, client=6)
    recs, n_seen = ag.agile_violation_list_read(log, lst)
    check(recs, n_seen, expected(addr, width, verdicts=ov, rids=orid), capacity)
    assert all(r.client == 6 for r in recs)
    # a fresh log has no list: the same check appends nothing, and reading is refused
    ag.agile_violation_log_init(log, 6)
    ag.agile_guard_check_batch(dev, d_addr, d_width, len(addr), d_v, log)
    with pytest.raises(ag.AgileError):
        ag.agile_violation_list_read(log, lst)


def test_list_aperture_check():
    ap = syn.table1_protected()
    addr, width, _ = syn.aperture_accesses(1 << 18)
    d_v = torch.empty(len(addr), dtype=torch.uint8, device=DEV)
    log = new_log()
    lst = new_list(log, 1 << 16)
    ag.agile_aperture_check_batch((ap.base, ap.size, ap.kind, ap.ident), to_dev(addr.view(np.int64)),
                                  to_dev(width), len(addr), d_v, log)
    ov, orid, olog = oracle.aperture_batch(ap, addr, width)
    assert (d_v.cpu().numpy() == ov).all()
    recs, n_seen = ag.agile_violation_list_read(log, lst)
    check(recs, n_seen, expected(addr, width, verdicts=ov, rids=orid), 1 << 16)


@pytest.mark.parametrize("op", ["copy", "triad"])
def test_list_stream(op):
    """Hand-fused streaming kernel on the hostile layout: every denied 16-byte unit and
    4-byte tail access, keyed by its address, with its site (b 0, c 1, a 1 or 2)."""
    n = 4099
    _, _, nbytes = _hostile_layout(n, 0)
    arena = torch.empty(nbytes, dtype=torch.uint8, device=DEV)
    base = arena.data_ptr()
    r, va, _ = _hostile_layout(n, base)
    _, dev = device_table(r, 12)
    b, c = _fill(n, 3)
    A, B, C = (arena[va[k] - base:va[k] - base + 4 * n].view(torch.float32) for k in "abc")
    B.copy_(torch.from_numpy(b))
    C.copy_(torch.from_numpy(c))
    log = new_log()
    lst = new_list(log, 8192)
    ag.agile_stream_launch(op, dev, A, B, C, n, 3.0, "poison", log)
    rc, rec = ag.agile_violation_log_read(log)
    _, olog = oracle.stream(op, r, va, b, c if op == "triad" else None, np.zeros(n, np.float32), 3.0)
    assert rec.count == olog.count
    arrays = [("b", 0)] + ([("c", 1)] if op == "triad" else []) + [("a", 2 if op == "triad" else 1)]
    n4 = n // 4
    a_l, w_l, s_l = [], [], []
    for name, site in arrays:
        a_l.append(va[name] + 16 * np.arange(n4, dtype=np.uint64)); w_l.append(np.full(n4, 16))
        s_l.append(np.full(n4, site))
        a_l.append(va[name] + 4 * np.arange(4 * n4, n, dtype=np.uint64)); w_l.append(np.full(n - 4 * n4, 4))
        s_l.append(np.full(n - 4 * n4, site))
    addr = np.concatenate(a_l).astype(np.uint64)
    width = np.concatenate(w_l).astype(np.uint8)
    sites = np.concatenate(s_l).astype(np.uint32)
    exp = expected(addr, width, sites, key_is_index=False, r=r)
    assert sum(exp.values()) == olog.count
    recs, n_seen = ag.agile_violation_list_read(log, lst)
    check(recs, n_seen, exp, 8192)


@pytest.mark.parametrize("kind", ["gather", "hist"])
def test_list_irregular(kind):
    """Hand-fused gather and histogram: the denied element and bin accesses, one entry
    each (a histogram bin hit by several keys appears that many times)."""
    from test_gpu_irregular import put, setup
    n = 40_003
    r, span, off, idx, key, bad, host, arena, base = setup(n, frac_bad=0.05)
    put(host, off["idx"], key if kind == "hist" else idx)
    t = r.shifted(base)
    _, dev = device_table(t, 16)
    arena.copy_(torch.from_numpy(host))
    log = new_log()
    lst = new_list(log, 1 << 14)
    target = off["bins"] if kind == "hist" else off["t"]
    ag.agile_irregular_launch(kind, dev, base + off["idx"], base + target, base + off["out"], n,
                              "poison", log)
    rc, rec = ag.agile_violation_log_read(log)
    va = {"t": base + target, "idx": base + off["idx"], "out": base + off["out"]}
    olog = oracle.irregular(kind, t, host.copy(), base, va, n, "poison")
    assert rec.count == olog.count
    ix = (key if kind == "hist" else idx).astype(np.int64)
    el_addr = (base + target + 4 * ix).astype(np.uint64)
    ev, erid, _ = oracle.check_batch(t, el_addr, np.full(n, 4, np.uint8), method="sorted")
    want = Counter((int(a), int(v), int(q)) for a, v, q in zip(el_addr[ev != 0], ev[ev != 0], erid[ev != 0]))
    assert sum(want.values()) == olog.count       # the only denials are element accesses
    recs, n_seen = ag.agile_violation_list_read(log, lst)
    assert n_seen == olog.count and len(recs) == olog.count
    assert Counter((r.addr, r.verdict, r.range_id) for r in recs) == want
    assert all(r.key == r.addr and r.width == 4 for r in recs)


def test_list_ptx_merged_at_every_exit():
    """The instrumented PTX kernel with early returns and exits: one entry per denied
    store, keyed by address, with its site; the register-merged log agrees."""
    n, m = 5000, 3333
    arena = torch.zeros(8 << 20, dtype=torch.uint8, device=DEV)
    a = arena.data_ptr() + 4096
    r = syn._ranges([a, a + 4 * m], [4 * m, 2 << 20], [0, 1], [7, 8])
    _, dev = device_table(r, 12)
    mod = ag.agile_module_load(ag.agile_guard_instrument_ptx(EXITS, "poison")[0])
    try:
        log = new_log()
        lst = new_list(log, 4096)
        ag.agile_module_bind(mod, dev, log)
        ag.agile_module_launch(mod, "agile_ptx_exits", (n + 255) // 256, 256,
                               [ctypes.c_uint64(a), ctypes.c_uint64(n)])
        rc, rec = ag.agile_violation_log_read(log)
        recs, n_seen = ag.agile_violation_list_read(log, lst)
    finally:
        mod.unload()
    i = np.arange(n, dtype=np.uint64)
    second = i[(i % 4 != 1) & (i % 4 != 2)]
    addr = np.concatenate([a + 4 * i, a + 4 * (second + 1)]).astype(np.uint64)
    sites = np.concatenate([np.zeros(n, np.uint32), np.ones(len(second), np.uint32)])
    exp = expected(addr, np.full(len(addr), 4, np.uint8), sites, key_is_index=False, r=r)
    assert rec.count == sum(exp.values())
    check(recs, n_seen, exp, 4096)


def test_list_batched_clients():
    """Many clients in one persistent launch, each log with a list of its own: every
    client's list holds the same multiset as when the client ran alone (whose count and
    first record the oracle fixes in the batched-launch tests)."""
    from paper_2606_06697_b300.clients import ClientSet
    from test_gpu_batch_clients import small_specs
    cs = ClientSet(small_specs(), DEV, log2_pages=(21,), frac_bad=0.01, policy="poison")
    n = len(cs.clients)
    cap = 1 << 14
    lists = [torch.zeros(ag.list_bytes(cap), dtype=torch.uint8, device=DEV) for _ in range(n)]

    def attach_all():
        for i in range(n):
            ag.agile_violation_list_attach(cs.log(i), lists[i], cap)

    cs.reset()
    attach_all()
    for i in range(n):
        cs.run_single(i, 0)
    alone = []
    for i in range(n):
        recs, seen = ag.agile_violation_list_read(cs.log(i), lists[i])
        _, rec = ag.agile_violation_log_read(cs.log(i))
        assert seen == rec.count == len(recs)
        alone.append(entries(recs))
    assert sum(sum(e.values()) for e in alone) > 0
    buf = torch.empty(ag.agile_batch_device_bytes(n), dtype=torch.uint8, device=DEV)
    cs.reset()
    attach_all()
    ag.agile_batch_upload(cs.work(0), 4096, buf)
    ag.agile_batch_launch(buf, n, 4096, True, 2)
    for i in range(n):
        recs, seen = ag.agile_violation_list_read(cs.log(i), lists[i])
        assert seen == sum(alone[i].values()) and entries(recs) == alone[i], i
