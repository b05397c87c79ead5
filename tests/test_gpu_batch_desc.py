"""Open-block descriptors of the batch check's second pass (windows under 4 GiB).

The uploaded descriptor slots are checked against blocks found here from the ranges
alone, with each descriptor's three verdicts taken from the oracle (one-byte accesses on
either side of the boundary, a two-byte access across it). Then the batch check is
compared with the oracle, verdict for verdict and log record for record, on tables dense
with boundaries of every kind pair, including one whose open blocks outnumber the slots.
The descriptor form runs for batches that give every lane of a full grid (one 1024-thread
block per SM) four groups of 8 accesses or more, so these batches are that large."""
import numpy as np
import pytest
import torch

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag
from gpu_util import DEV, assert_log_equal, device_table, new_log, to_dev
from test_gpu_batch import run_batch
from test_gpu_table import block_classes

pytestmark = pytest.mark.gpu

EMPTY = 0xFFFFFFFF


def desc_batch():
    """Accesses in the smallest batch that takes the descriptor form, plus a ragged 3."""
    return 4 * 8 * 1024 * torch.cuda.get_device_properties(0).multi_processor_count + 3


def dense_table(n, seed, base=0x7F3A00000000):
    """n ranges of 1 B to 16 KiB, a third abutting the one before, the rest after gaps
    of 1 B to 16 KiB; kinds 4:2:1 user, protected, MMIO."""
    st = syn.Stream(seed, 1)
    size = st.log_uniform(1, 1 << 14, n)
    gap = np.where(st.below(3, n) == 0, 0, st.log_uniform(1, 1 << 14, n))
    start = base + np.cumsum(gap + size) - size
    kind = st.choice(np.array([0, 0, 0, 0, 1, 1, 2], np.uint32), n)
    return syn._ranges(start.astype(np.uint64), size, kind, np.arange(n) + 100)


def top_table():
    """Two ranges in the last 8 KiB of the address space: the last block ends at 2^64."""
    return syn._ranges(np.array([2**64 - 8192, 2**64 - 4096], dtype=np.uint64),
                       np.array([4000, 4095], dtype=np.uint64), [0, 2], [1, 2])


def expected_descs(r, lo, clg, cn):
    """{block: payload} for every open block with at most one range edge strictly inside
    it, the block ending at 2^64 excepted."""
    C = 1 << clg
    cls = block_classes(r, lo, clg, cn)[:cn]
    ks = np.flatnonzero(cls == 0).astype(np.uint64)
    s = np.uint64(lo) + ks * np.uint64(C)
    keep = s <= np.uint64(2**64 - 1 - C)                  # s + C representable
    ks, s = ks[keep], s[keep]
    edges = np.unique(np.concatenate([r.base, r.base + r.size]).astype(np.uint64))
    i0 = np.searchsorted(edges, s, side="right")
    i1 = np.searchsorted(edges, s + np.uint64(C), side="left")
    one = i1 - i0 <= 1
    ks, s, i0, has = ks[one], s[one], i0[one], (i1 - i0)[one] == 1
    p = np.where(has, edges[np.minimum(i0, len(edges) - 1)], s + np.uint64(C))
    one_b = np.ones(len(s), np.uint8)
    vl, _, _ = oracle.check_batch(r, s, one_b, method="sorted")
    vr, _, _ = oracle.check_batch(r, np.where(has, p, s), one_b, method="sorted")
    vs, _, _ = oracle.check_batch(r, np.where(has, p - np.uint64(1), s), one_b + 1, method="sorted")
    pay = (p - s).astype(np.uint64) | vl.astype(np.uint64) << 16 | vr.astype(np.uint64) << 20 | \
        vs.astype(np.uint64) << 24
    return dict(zip(ks.tolist(), pay.tolist()))


def slot_of(k, K, lg):
    return ((k * K) & 0xFFFFFFFF) >> (32 - lg)


def device_slots(dev):
    v = dev.view
    img = dev.buf.cpu().numpy()
    off = v.cdesc - dev.address
    return img[off:off + (8 << v.cdesc_log2)].view(np.uint32).reshape(-1, 2)


@pytest.mark.parametrize("name", ["batch", "dense", "dense_many", "top"])
def test_descriptor_slots(name):
    r = {"batch": syn.batch_table, "dense": lambda: dense_table(800, 5),
         "dense_many": lambda: dense_table(6000, 6), "top": top_table}[name]()
    for lg_page in (12, 21):
        _, dev = device_table(r, lg_page)
        v = dev.view
        assert v.cdesc and 6 <= v.cdesc_log2 <= 12
        want = expected_descs(r, v.lo, v.cmap_log2, v.cmap_n)
        slots = device_slots(dev)
        held = {}
        for j, (k, pay) in enumerate(slots.tolist()):
            if k == EMPTY:
                continue
            assert k not in held and k in want, (name, k)
            assert j in (slot_of(k, v.cdesc_k1, v.cdesc_log2), slot_of(k, v.cdesc_k2, v.cdesc_log2))
            assert pay == want[k], (name, k, hex(pay), hex(want[k]))
            held[k] = pay
        if 4 * len(want) <= 1 << v.cdesc_log2:
            assert len(held) == len(want), (name, len(held), len(want))   # every one placed
        else:
            assert len(held) > (1 << v.cdesc_log2) // 4                  # the slots fill up
        if name == "top":
            assert all(v.lo + (k + 1) * (1 << v.cmap_log2) < 2**64 for k in held)


def edge_accesses(r, n, seed):
    """Accesses within 32 bytes of a range edge, widths legal and not, plus a few below,
    beyond and far from the window."""
    st = syn.Stream(seed, 2)
    edges = np.concatenate([r.base, r.base + r.size]).astype(np.int64)
    a = edges[st.below(len(edges), n)] + st.below(64, n) - 32
    lo, hi = int(r.base.min()), int((r.base + r.size).max())
    m = n // 64
    a[:m] = lo - st.below(1 << 16, m) - 1
    a[m:2 * m] = hi + st.below(1 << 16, m)
    a[2 * m:3 * m] = st.below(1 << 40, m)
    w = st.choice(np.array([1, 2, 4, 8, 16, 1, 2, 4, 8, 16, 0, 3, 32], np.uint8), n)
    return a.astype(np.uint64), w


@pytest.mark.parametrize("n_ranges,seed", [(800, 5), (6000, 6), (3000, 7)])
@pytest.mark.parametrize("lg_page", [12, 21])
def test_batch_parity_dense_boundaries(n_ranges, seed, lg_page):
    r = dense_table(n_ranges, seed)
    addr, width = edge_accesses(r, desc_batch(), seed)
    _, dev = device_table(r, lg_page)
    v, rc, rec = run_batch(dev, addr, width, client=3)
    ov, _, olog = oracle.check_batch(r, addr, width, method="sorted")
    assert (v == ov).all(), np.flatnonzero(v != ov)[:10]
    for verdict in range(6):                               # every verdict occurs
        assert (ov == verdict).any(), verdict
    assert_log_equal(rec, olog, client=3)


@pytest.mark.parametrize("lg_page", [12, 16, 21])
def test_batch_parity_workload_descriptor_form(lg_page):
    """The batch workload repeated to the descriptor form's size: at 4 KiB and 64 KiB pages
    the page map does not fit in shared memory beside the class map, descriptors and
    queue, and the form without the staged page map runs."""
    t = syn.batch_table()
    addr, width, label = syn.batch_accesses(t, 1 << 20)
    m = desc_batch()
    reps = -(-m // len(addr))
    addr, width, label = (np.tile(x, reps)[:m] for x in (addr, width, label))
    tbl, dev = device_table(t, lg_page)
    if lg_page == 12:
        assert tbl.geometry()[1] * 4 > 96 * 1024          # the page map alone is 1 MiB
    v, rc, rec = run_batch(dev, addr, width, client=4)
    assert (v == label).all()
    _, _, olog = oracle.check_batch(t, addr[:1 << 20], width[:1 << 20], method="sorted")
    assert rec.count == int((label != 0).sum())
    assert (rec.key, rec.addr, rec.width, rec.verdict, rec.range_id) == \
        (olog.key, olog.addr, olog.width, olog.verdict, olog.range_id)


def test_batch_parity_descriptor_first_record():
    """The smallest denied index decided by a descriptor: the log's first record carries
    the range id the full rule finds."""
    r = dense_table(800, 9)
    addr, width = edge_accesses(r, desc_batch(), 9)
    _, dev = device_table(r, 21)
    v = dev.view
    want = expected_descs(r, v.lo, v.cmap_log2, v.cmap_n)
    ov, orid, _ = oracle.check_batch(r, addr, width, method="sorted")
    # the first straddle inside one described block goes first
    off = addr.astype(np.uint64) - np.uint64(v.lo)
    blk = (off >> np.uint64(v.cmap_log2)).astype(np.int64)
    inblk = (off & np.uint64((1 << v.cmap_log2) - 1)) + width <= (1 << v.cmap_log2)
    described = np.array([b in want for b in blk.tolist()]) & inblk & (off < np.uint64(1 << 32))
    j = int(np.flatnonzero((ov == 3) & described)[0])
    order = np.r_[j, np.delete(np.arange(len(addr)), j)]
    addr, width = addr[order], width[order]
    v, rc, rec = run_batch(dev, addr, width)
    ov, orid, olog = oracle.check_batch(r, addr, width, method="sorted")
    assert (v == ov).all()
    assert olog.key == 0 and olog.verdict == 3 and olog.range_id != 0xFFFFFFFF
    assert_log_equal(rec, olog)


def test_batch_parity_all_open():
    """Nearly every access open: a window of MMIO ranges with an allocation after every
    seventh, so pass 1 decides only the accesses inside allocations (a tenth), and each
    warp's round of groups has more open accesses than its list holds (the owner search
    deals them)."""
    base = 0x7E5500000000
    n = 4096
    st = syn.Stream(77, 3)
    size = np.full(n, 8192, np.int64)
    start = base + np.arange(n, dtype=np.int64) * 8192
    kind = np.where(np.arange(n) % 8 == 7, syn.KIND_USER, syn.KIND_MMIO).astype(np.uint32)
    r = syn._ranges(start.astype(np.uint64), size, kind, np.arange(n) + 1)
    m = desc_batch()
    a = (base + st.below(n * 8192 + 4096, m) - 2048).astype(np.uint64)
    w = st.choice(np.array([1, 2, 4, 8, 16, 3], np.uint8), m)
    _, dev = device_table(r, 21)
    v, rc, rec = run_batch(dev, a, w, client=9)
    ov, _, olog = oracle.check_batch(r, a, w, method="sorted")
    assert (v == ov).all(), np.flatnonzero(v != ov)[:10]
    assert (ov == 2).mean() > 0.7                        # MMIO
    assert_log_equal(rec, olog, client=9)


@pytest.mark.parametrize("size", ["1M", "descriptor form"])
def test_log_accumulates_over_launches(size):
    """Two checks into one log, in either order: the count is the sum, and the first record
    is the one with the smaller key, whichever launch found it (the log merge lowers the
    key word first and lets only the lowering blocks write the record)."""
    t = syn.batch_table()
    addr, width, label = syn.batch_accesses(t, 1 << 20)
    m = (1 << 20) if size == "1M" else desc_batch()
    reps = -(-m // len(addr))
    y_a, y_w = (np.tile(x, reps)[:m] for x in (addr, width))
    ok = int(np.flatnonzero(label == 0)[0])
    x_a, x_w = y_a.copy(), y_w.copy()
    x_a[:5000], x_w[:5000] = addr[ok], width[ok]       # X's first violation comes later
    _, ox = oracle.check_batch(t, x_a, x_w, method="sorted")[::2]
    _, oy = oracle.check_batch(t, y_a, y_w, method="sorted")[::2]
    assert oy.key < ox.key
    _, dev = device_table(t, 21)
    d_v = torch.empty(m, dtype=torch.uint8, device=DEV)
    for order in ((x_a, x_w), (y_a, y_w)), ((y_a, y_w), (x_a, x_w)):
        log = new_log(client=2)
        for a, w in order:
            ag.agile_guard_check_batch(dev, to_dev(a.view(np.int64)), to_dev(w), m, d_v, log)
        rc, rec = ag.agile_violation_log_read(log)
        assert rec.count == ox.count + oy.count
        assert (rec.key, rec.addr, rec.width, rec.verdict, rec.range_id) == \
            (oy.key, oy.addr, oy.width, oy.verdict, oy.range_id)


def test_batch_parity_top_of_address_space():
    """The descriptor form on a window that ends at 2^64: accesses over its last blocks,
    widths legal and not, some ending past 2^64 - 1 (INVALID); the block that ends at 2^64
    has no descriptor and its accesses reach the full rule."""
    r = top_table()
    m = desc_batch()
    st = syn.Stream(91, 4)
    a = (np.uint64(2**64 - 12288) + st.below(12288, m).astype(np.uint64)).astype(np.uint64)
    w = st.choice(np.array([1, 2, 4, 8, 16, 0, 3, 32], np.uint8), m)
    for lg_page in (12, 21):
        _, dev = device_table(r, lg_page)
        v, rc, rec = run_batch(dev, a, w, client=8)
        ov, _, olog = oracle.check_batch(r, a, w, method="sorted")
        assert (v == ov).all(), np.flatnonzero(v != ov)[:10]
        assert (ov == 5).any() and (ov == 0).any() and (ov == 2).any()
        assert_log_equal(rec, olog, client=8)
