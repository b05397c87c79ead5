"""Batch guard check on the GPU vs the oracle: verdicts and log, bit for bit."""
import numpy as np
import pytest
import torch

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag
from gpu_util import DEV, assert_log_equal, device_table, new_log, to_dev

pytestmark = pytest.mark.gpu


def run_batch(dev, addr, width, offset=0, client=0):
    """Device check; `offset` shifts the device arrays off their natural alignment."""
    n = len(addr)
    a_buf = torch.zeros(n + 2, dtype=torch.int64, device=DEV)
    w_buf = torch.zeros(n + 16, dtype=torch.uint8, device=DEV)
    v_buf = torch.full((n + 16,), 0xEE, dtype=torch.uint8, device=DEV)
    if n:
        a_buf[offset:offset + n] = to_dev(addr.view(np.int64))
        w_buf[offset:offset + n] = to_dev(width)
    log = new_log(client)
    ag.agile_guard_check_batch(dev, a_buf.data_ptr() + 8 * offset, w_buf.data_ptr() + offset, n,
                               v_buf.data_ptr() + offset, log)
    rc, rec = ag.agile_violation_log_read(log)
    v = v_buf.cpu().numpy()
    assert (v[:offset] == 0xEE).all() and (v[offset + n:] == 0xEE).all()   # no stray writes
    return v[offset:offset + n], rc, rec


@pytest.mark.parametrize("log2_page", [16, 21])
def test_batch_workload_full(log2_page):
    """The 1M-access batch workload: 84 ranges in a 1 GiB window."""
    t = syn.batch_table()
    addr, width, label = syn.batch_accesses(t, 1 << 20)
    _, dev = device_table(t, log2_page)
    v, rc, rec = run_batch(dev, addr, width, client=7)
    ov, _, olog = oracle.check_batch(t, addr, width, method="sorted")
    assert (v == ov).all()
    assert (v == label).all()
    assert rc == 1
    assert_log_equal(rec, olog, client=7)


@pytest.mark.parametrize("n", [0, 1, 7, 8, 9, 255, 4097, 100_003])
@pytest.mark.parametrize("offset", [0, 1])
def test_batch_ragged_and_misaligned(n, offset):
    t = syn.batch_table(seed=12345)
    addr, width, _ = syn.batch_accesses(t, max(n, 1), seed=99)
    addr, width = addr[:n], width[:n]
    _, dev = device_table(t, 21)
    v, rc, rec = run_batch(dev, addr, width, offset=offset)
    ov, _, olog = oracle.check_batch(t, addr, width, method="sorted")
    assert (v == ov).all()
    assert_log_equal(rec, olog)


def test_batch_table1_global_map():
    """Table I's 1.5 TiB window has too many pages for shared memory: global map path."""
    t = syn.table1_apertures()
    tbl, dev = device_table(t, 21)
    assert tbl.geometry()[1] * 4 > 48 * 1024
    st = syn.Stream(21, 1)
    edges = np.array([*syn.TABLE1_MMIO, syn.TABLE1_PROTECTED[1], syn.TABLE1_USER[1]], np.int64)
    n = 50_000
    a = (edges[st.below(4, n)] + st.below(1 << 22, n) - (1 << 21)).astype(np.uint64)
    w = st.choice(np.array([0, 1, 2, 3, 4, 8, 16, 32], np.uint8), n)
    v, _, rec = run_batch(dev, a, w)
    ov, _, olog = oracle.check_batch(t, a, w, method="sorted")
    assert (v == ov).all()
    assert_log_equal(rec, olog)


def test_batch_tiny_tables_exhaustive():
    """Tiny tables (<= 6 ranges, abutting and gapped) at 4 KiB pages, every address x
    width around them, including the top of the address space."""
    for lo in (0x10000 - 96, 2**64 - 4096):
        st = syn.Stream(31, lo & 0xFFFF)
        for trial in range(12):
            k = int(st.below(7, 1)[0])
            cuts = np.sort(st.below(192, 2 * k))
            base, size, kind = [], [], []
            for i in range(k):
                b0, b1 = int(cuts[2 * i]), int(cuts[2 * i + 1])
                if b1 > b0:
                    base.append(lo + b0)
                    size.append(b1 - b0)
                    kind.append(int(st.below(3, 1)[0]))
            t = syn._ranges(base, size, kind, list(range(50, 50 + len(base))))
            _, dev = device_table(t, 12)
            aa = np.arange(max(lo - 24, 0), min(lo + 220, 2**64 - 1), dtype=np.uint64)
            ws = np.array([1, 2, 3, 4, 8, 16], np.uint8)
            addr = np.repeat(aa, len(ws))
            width = np.tile(ws, len(aa))
            v, _, rec = run_batch(dev, addr, width)
            ov, _, olog = oracle.check_batch(t, addr, width, method="linear")
            assert (v == ov).all()
            assert_log_equal(rec, olog)


def test_batch_empty_table_and_edges():
    t = syn._ranges([], [], [], [])
    _, dev = device_table(t, 21)
    addr = np.array([0, 1, 2**64 - 16, 2**64 - 17, 2**63], np.uint64)
    width = np.array([1, 0, 16, 16, 8], np.uint8)
    v, rc, rec = run_batch(dev, addr, width)
    ov, _, olog = oracle.check_batch(t, addr, width)
    assert (v == ov).all() and rc == 1
    assert_log_equal(rec, olog)


def test_batch_no_violation_log_empty():
    t = syn.batch_table()
    addr, width, label = syn.batch_accesses(t, 20_000, frac_deny_in=0, frac_straddle=0,
                                            frac_unmapped=0)
    _, dev = device_table(t, 21)
    v, rc, rec = run_batch(dev, addr, width)
    assert (v == 0).all() and rc == 0 and rec.count == 0 and rec.range_id == ag.NO_RANGE


@pytest.mark.parametrize("log2_page", [12, 16, 21])
def test_batch_full_size_as_benchmarked(log2_page):
    """2^28 checks, the benchmark's input (1M generated accesses repeated): every verdict
    equals its access's generator label, and the log holds the first denial and the
    exact count."""
    t = syn.batch_table()
    m, n = 1 << 20, 1 << 28
    addr, width, label = syn.batch_accesses(t, m)
    _, dev = device_table(t, log2_page)
    da = torch.from_numpy(addr.view(np.int64)).to(DEV).repeat(n // m)
    dw = torch.from_numpy(width).to(DEV).repeat(n // m)
    dv = torch.empty(n, dtype=torch.uint8, device=DEV)
    log = new_log()
    ag.agile_guard_check_batch(dev, da, dw, n, dv, log)
    rc, rec = ag.agile_violation_log_read(log)
    lab = torch.from_numpy(label).to(DEV)
    assert torch.equal(dv.view(n // m, m), lab.expand(n // m, m))
    first = int(np.flatnonzero(label)[0])
    assert rc == 1 and rec.count == (n // m) * int((label != 0).sum())
    assert (rec.key, rec.addr, rec.width, rec.verdict) == \
        (first, int(addr[first]), int(width[first]), int(label[first]))
