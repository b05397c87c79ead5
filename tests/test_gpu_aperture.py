"""Aperture-only batch check on the GPU vs the oracle's aperture rule, bit for bit."""
import os

import numpy as np
import pytest
import torch

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag
from gpu_util import DEV, assert_log_equal, new_log, to_dev

pytestmark = pytest.mark.gpu
V = {name: i for i, name in enumerate(oracle.VERDICT_NAMES)}


def aps(r):
    return (r.base, r.size, r.kind, r.ident)


def run(r, addr, width, offset=0, client=0):
    n = len(addr)
    a_buf = torch.zeros(n + 2, dtype=torch.int64, device=DEV)
    w_buf = torch.zeros(n + 16, dtype=torch.uint8, device=DEV)
    v_buf = torch.full((n + 16,), 0xEE, dtype=torch.uint8, device=DEV)
    if n:
        a_buf[offset:offset + n] = to_dev(addr.view(np.int64))
        w_buf[offset:offset + n] = to_dev(width)
    log = new_log(client)
    ag.agile_aperture_check_batch(aps(r), a_buf.data_ptr() + 8 * offset, w_buf.data_ptr() + offset,
                                  n, v_buf.data_ptr() + offset, log)
    rc, rec = ag.agile_violation_log_read(log)
    v = v_buf.cpu().numpy()
    assert (v[:offset] == 0xEE).all() and (v[offset + n:] == 0xEE).all()
    return v[offset:offset + n], rc, rec


def test_aperture_table1_golden():
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table1_aperture_rule.txt")):
        f = line.split()
        if f and not f[0].startswith("#"):
            rows.append((int(f[1], 16), int(f[2], 0), V[f[3]]))
    addr = np.array([x[0] for x in rows], dtype=np.uint64)
    width = np.array([x[1] for x in rows], dtype=np.uint8)
    v, rc, rec = run(syn.table1_protected(), addr, width, client=3)
    assert v.tolist() == [x[2] for x in rows]
    _, _, olog = oracle.aperture_batch(syn.table1_protected(), addr, width)
    assert_log_equal(rec, olog, client=3)


@pytest.mark.parametrize("n", [0, 1, 7, 9, 4097, 1 << 20])
@pytest.mark.parametrize("offset", [0, 1])
def test_aperture_workload(n, offset):
    addr, width, label = syn.aperture_accesses(max(n, 1))
    addr, width, label = addr[:n], width[:n], label[:n]
    v, rc, rec = run(syn.table1_protected(), addr, width, offset=offset)
    ov, _, olog = oracle.aperture_batch(syn.table1_protected(), addr, width)
    assert (v == ov).all() and (v == label).all()
    assert_log_equal(rec, olog)


def test_aperture_four_apertures_tiny_windows():
    """Four apertures (two MMIO, two protected) in a small window; every address and
    width around them, against the oracle."""
    r = syn._ranges([0x1000, 0x1040, 0x10A0, 0x1100], [0x40, 0x30, 0x10, 0x8],
                    [syn.KIND_PROTECTED, syn.KIND_MMIO, syn.KIND_PROTECTED, syn.KIND_MMIO],
                    [7, 8, 9, 10])
    a = np.repeat(np.arange(0xFF0, 0x1120, dtype=np.uint64), 6)
    w = np.tile(np.array([1, 2, 3, 4, 8, 16], dtype=np.uint8), 0x1120 - 0xFF0)
    v, rc, rec = run(r, a, w)
    ov, _, olog = oracle.aperture_batch(r, a, w)
    assert (v == ov).all()
    assert_log_equal(rec, olog)


def test_aperture_full_size_against_labels():
    """2^28 accesses (2.4 GB in, 268 MB out) against the generator's labels."""
    n = 1 << 28
    addr, width, label = syn.aperture_accesses(n)
    d_a = torch.from_numpy(addr.view(np.int64)).to(DEV)
    d_w = torch.from_numpy(width).to(DEV)
    d_v = torch.empty(n, dtype=torch.uint8, device=DEV)
    log = new_log()
    ag.agile_aperture_check_batch(aps(syn.table1_protected()), d_a, d_w, n, d_v, log)
    rc, rec = ag.agile_violation_log_read(log)
    assert torch.equal(d_v.cpu(), torch.from_numpy(label))
    first = int(np.flatnonzero(label)[0])
    assert rc == 1 and rec.count == int((label != 0).sum()) and rec.key == first
    assert (rec.addr, rec.width, rec.verdict) == (int(addr[first]), int(width[first]), int(label[first]))
