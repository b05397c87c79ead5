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


def run_case(kind, policy, n, log2_page, fast_path="bitmap", **kw):
    r, span, off, idx, key, bad, host, arena, base = setup(n, **kw)
    put(host, off["idx"], key if kind == "hist" else idx)
    t = r.shifted(base)
    _, dev = device_table(t, log2_page)
    arena.copy_(torch.from_numpy(host))
    log = new_log(client=4)
    target = off["bins"] if kind == "hist" else off["t"]
    ag.agile_irregular_launch_fastpath(kind, dev, base + off["idx"], base + target,
                                       base + off["out"], n, policy, log, fast_path)
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


@pytest.mark.parametrize("kind", ["gather", "scatter", "hist"])
@pytest.mark.parametrize("n", [131, 40_003])
def test_irregular_match_fast_path(kind, n):
    """The __match_any_sync form of the per-lane bitmap read decides exactly as the
    per-lane form: outputs and log equal the oracle's (ragged last group included)."""
    run_case(kind, "poison", n, 16, fast_path="match", frac_bad=0.05)
    run_case(kind, "poison", n, 16, fast_path="match", dist="zipf", stripes=64, seed=9)


def test_irregular_match_fast_path_arguments():
    with pytest.raises(ag.AgileError):         # the match form is built for POISON only
        ag.agile_irregular_launch_fastpath("gather", None, 0x1000, 0x2000, 0x3000, 64, "poison",
                                           None, "match")


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


# ---------------------------------------------------------------- REMAP_OR


def remap_setup(n, half=1 << 20, seed=6):
    """remap_layout in a device arena aligned to 2 * half (the mask's block)."""
    r, span, off = syn.remap_layout(n, half)
    idx, key, cls = syn.remap_indices(n, half, seed=syn.SEED_BASE + seed)
    host = np.zeros(span, np.uint8)
    host[:2 * half] = syn.Stream(6, 7).uniform(half // 2).astype(np.float32).view(np.uint8)
    raw = torch.empty(span + 2 * half, dtype=torch.uint8, device=DEV)
    skew = (-raw.data_ptr()) % (2 * half)
    arena = raw[skew:skew + span]
    return r, off, idx, key, cls, host, arena, arena.data_ptr()


def remap_table(r, base, half, log2_page):
    s = r.shifted(base)
    t = ag.agile_guard_table_build(s.base, s.size, s.kind, s.ident, log2_page)
    t.set_remap(half)
    buf = torch.empty(t.device_bytes(), dtype=torch.uint8, device=DEV)
    return t, t.upload(buf)


@pytest.mark.parametrize("kind", ["gather", "scatter", "hist"])
@pytest.mark.parametrize("log2_page", [12, 21])
@pytest.mark.parametrize("n", [5, 40_003])
def test_irregular_remap_parity(kind, log2_page, n):
    half = 1 << 20
    r, off, idx, key, cls, host, arena, base = remap_setup(n, half)
    put(host, off["idx"], key if kind == "hist" else idx)
    _, dev = remap_table(r, base, half, log2_page)
    arena.copy_(torch.from_numpy(host))
    log = new_log(client=7)
    target = off["bins"] if kind == "hist" else off["t"]
    ag.agile_irregular_launch(kind, dev, base + off["idx"], base + target,
                              base + off["out"], n, "remap", log)
    rc, rec = ag.agile_violation_log_read(log)
    va = {"t": base + target, "idx": base + off["idx"], "out": base + off["out"]}
    olog = oracle.irregular(kind, r.shifted(base), host, base, va, n, "remap", remap=half)
    assert_remap_arena(kind, arena.cpu().numpy(), host, off, idx, cls, half)
    assert_log_equal(rec, olog, client=7)


def assert_remap_arena(kind, got, want, off, idx, cls, half):
    """Arena vs the oracle's. A scatter element that a remapped access and a direct one
    both write gets either value (the kernels run in parallel; the oracle in index order),
    so those elements are checked against the two candidates and the rest bit for bit."""
    if kind != "scatter":
        assert (got == want).all(), kind
        return
    ne = half // 4
    both = np.intersect1d(idx[cls == 1] + ne, idx[cls == 0])
    t = got[off["t"]:off["t"] + 4 * ne].view(np.float32)
    direct = (both & 0xFFFFFF).astype(np.float32)
    moved = ((both - ne).astype(np.uint64) & np.uint64(0xFFFFFF)).astype(np.float32)
    assert ((t[both] == direct) | (t[both] == moved)).all()
    got = got.copy()
    got[off["t"]:off["t"] + 4 * ne].view(np.float32)[both] = \
        want[off["t"]:off["t"] + 4 * ne].view(np.float32)[both]
    assert (got == want).all(), kind


def test_remap_policy_refused_where_unsupported():
    """The streaming kernels and batched work items take poison, sink and report only."""
    r, off, idx, key, cls, host, arena, base = remap_setup(64)
    _, dev = remap_table(r, base, 1 << 20, 21)
    x = arena[off["out"]:off["out"] + 256].view(torch.float32)
    with pytest.raises(ag.AgileError):
        ag.agile_stream_launch("copy", dev, x, x, None, 64, 1.0, "remap")


@pytest.mark.parametrize("kind", ["gather", "scatter", "hist"])
@pytest.mark.parametrize("log2_page", [12, 16])
def test_irregular_stress_layout(kind, log2_page):
    """The adversarial 60 KiB user + 4 KiB protected stripes: with 64 KiB pages and
    bitmap blocks no page is all user, so every element takes the full classification."""
    run_case(kind, "poison", 40_003, log2_page, stripes=256, user=60 * 1024, prot=4 * 1024,
             bins=1 << 10, frac_bad=0.01)
