"""Guarded gather / scatter / histogram on the GPU vs the oracle, bit for bit."""
import numpy as np
import pytest
import torch

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag
from gpu_util import DEV, assert_log_equal, device_table, new_log

pytestmark = pytest.mark.gpu


def setup(n, stripes=16, user=64 * 1024, prot=4 * 1024, bins=1 << 12, frac_bad=0.01,
          dist="uniform", seed=5):
    r, span, off = syn.irregular_layout(n, stripes, user, prot, bins)
    idx, key, bad = syn.irregular_indices(n, stripes, user, prot, bins, dist=dist,
                                          frac_bad=frac_bad, seed=seed)
    host = np.zeros(span, np.uint8)
    st = syn.Stream(6, 6)
    tv = st.uniform((stripes * (user + prot)) // 4).astype(np.float32)
    host[:len(tv) * 4] = tv.view(np.uint8)
    dev_arena = torch.empty(span, dtype=torch.uint8, device=DEV)
    base = dev_arena.data_ptr()
    return r, span, off, idx, key, bad, host, dev_arena, base


def put(host, off, arr):
    b = np.ascontiguousarray(arr).view(np.uint8)
    host[off:off + len(b)] = b


def run_case(kind, policy, n, log2_page, **kw):
    r, span, off, idx, key, bad, host, arena, base = setup(n, **kw)
    put(host, off["idx"], key if kind == "hist" else idx)
    t = r.shifted(base)
    _, dev = device_table(t, log2_page)
    arena.copy_(torch.from_numpy(host))
    log = new_log(client=4)
    target = off["bins"] if kind == "hist" else off["t"]
    ag.agile_irregular_launch(kind, dev, base + off["idx"], base + target,
                              base + off["out"], n, policy, log)
    rc, rec = ag.agile_violation_log_read(log)
    got = arena.cpu().numpy()
    va = {"t": base + target, "idx": base + off["idx"], "out": base + off["out"]}
    olog = oracle.irregular(kind, t, host, base, va, n, policy)
    assert (got == host).all(), (kind, policy)
    assert_log_equal(rec, olog, client=4)
    assert rc == (1 if olog.count else 0)


@pytest.mark.parametrize("kind", ["gather", "scatter", "hist"])
@pytest.mark.parametrize("policy", ["poison", "sink", "report"])
@pytest.mark.parametrize("log2_page", [12, 16, 21])
def test_irregular_parity(kind, policy, log2_page):
    run_case(kind, policy, 40_003, log2_page)


@pytest.mark.parametrize("kind", ["gather", "scatter", "hist"])
def test_irregular_zipf(kind):
    run_case(kind, "poison", 100_000, 16, dist="zipf", stripes=64)


@pytest.mark.parametrize("n", [1, 3, 4, 5, 131])
def test_irregular_ragged(n):
    for kind in ("gather", "scatter", "hist"):
        run_case(kind, "poison", n, 21, frac_bad=0.5)


def test_irregular_no_violation_matches_unguarded():
    n = 1 << 20
    r, span, off, idx, key, bad, host, arena, base = setup(n, frac_bad=0)
    put(host, off["idx"], idx)
    _, dev = device_table(r.shifted(base), 21)
    arena.copy_(torch.from_numpy(host))
    out = arena[off["out"]:off["out"] + 4 * n].view(torch.float32)
    log = new_log()
    ag.agile_irregular_launch("gather", dev, base + off["idx"], base, out, n, "poison", log)
    g = out.clone()
    out.zero_()
    ag.agile_irregular_launch("gather", None, base + off["idx"], base, out, n)
    rc, rec = ag.agile_violation_log_read(log)
    assert rc == 0 and torch.equal(g, out)
    tv = host[:16 * (64 + 4) * 1024].view(np.float32)
    assert (g.cpu().numpy() == tv[idx]).all()


def test_irregular_full_size_gather_uniform():
    """2^28 int64 indices into the 16 GiB striped table (4096 x 4 MiB user ranges, each
    followed by a 64 KiB protected range); 0.1% aimed into the protected ranges. Guarded
    output equals the unguarded one except at those positions, which read 0; the log
    counts them and names the lowest-addressed one."""
    n = 1 << 28
    r, span, off = syn.irregular_layout(n)
    idx, key, bad = syn.irregular_indices(n)
    arena = torch.empty(span, dtype=torch.uint8, device=DEV)
    base = arena.data_ptr()
    tview = arena[:off["bins"]].view(torch.float32)
    tview.uniform_(1, 2)
    d_idx = arena[off["idx"]:off["idx"] + 8 * n].view(torch.int64)
    d_idx.copy_(torch.from_numpy(idx))
    out = arena[off["out"]:off["out"] + 4 * n].view(torch.float32)
    for lg in (21, 16):
        _, dev = device_table(r.shifted(base), lg)
        log = new_log()
        ag.agile_irregular_launch("gather", dev, d_idx, base, out, n, "poison", log)
        rc, rec = ag.agile_violation_log_read(log)
        g = out.clone()
        ag.agile_irregular_launch("gather", None, d_idx, base, out, n)
        d_bad = torch.from_numpy(bad).to(DEV)
        assert torch.equal(g[~d_bad], out[~d_bad]) and bool((g[d_bad] == 0).all())
        assert rc == 1 and rec.count == int(bad.sum())
        first = base + 4 * int(idx[bad].min())
        assert (rec.key, rec.addr, rec.site, rec.width, rec.verdict) == (first, first, 2, 4, 1)
        del g
