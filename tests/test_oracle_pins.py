"""Pins for the oracle: checks against facts fixed outside the oracle itself.

- Table I golden cases derived by hand (tests/golden/table1_apertures.txt), and for the
  aperture rule (tests/golden/table1_aperture_rule.txt).
- Brute force on tiny tables through a per-byte ownership formulation: every byte of a
  small window is assigned its owning range, and the verdict is read off the set of
  owners -- a different computation from the oracle's interval compares.
- The Table I special case as a closed form of four compares.
- Generator labels: the batch workload's accesses are placed by construction, so the
  verdict histogram is known exactly.
- IEEE arithmetic of the reference kernels: scale is one rounded multiply, triad one
  correctly rounded fused multiply-add, checked with exact rationals.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import agile_synth as syn
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_apertures.txt")
V = {name: i for i, name in enumerate(oracle.VERDICT_NAMES)}
M64 = 2**64 - 1


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        rows.append((f[0], int(f[1], 16), int(f[2], 0), V[f[3]], int(f[4], 16)))
    return rows


@pytest.mark.parametrize("method", ["linear", "sorted"])
def test_table1_golden_batch(method):
    rows = [r for r in _golden_rows() if r[0] == "b"]
    t = syn.table1_apertures()
    addr = np.array([r[1] for r in rows], dtype=np.uint64)
    width = np.array([r[2] for r in rows], dtype=np.uint8)
    v, rid, log = oracle.check_batch(t, addr, width, method=method)
    assert v.tolist() == [r[3] for r in rows]
    assert rid.tolist() == [r[4] for r in rows]
    first = next(i for i, r in enumerate(rows) if r[3] != 0)
    assert log.key == first and log.count == sum(r[3] != 0 for r in rows)


def test_table1_golden_validate():
    rows = [r for r in _golden_rows() if r[0] == "v"]
    t = syn.table1_apertures()
    v, rid = oracle.validate(t, np.array([r[1] for r in rows], dtype=np.uint64),
                             np.array([r[2] for r in rows], dtype=np.uint64))
    assert v.tolist() == [r[3] for r in rows]
    assert rid.tolist() == [r[4] for r in rows]


def test_table1_closed_form():
    """Table I: three abutting apertures, so the rule is four interval compares."""
    (m0, m1), (p0, p1), (u0, u1) = syn.TABLE1_MMIO, syn.TABLE1_PROTECTED, syn.TABLE1_USER
    st = syn.Stream(7, 99)
    edges = np.array([m0, m1, p1, u1], dtype=np.int64)
    n = 20000
    a = edges[st.below(4, n)] + st.below(64, n) - 32
    w = st.choice(syn.WIDTHS, n).astype(np.int64)
    exp = np.full(n, V["UNMAPPED"])
    e = a + w
    exp[(a < u1) & (e > p1)] = V["STRADDLE"]
    exp[(a < p1) & (e > m1)] = V["PROTECTED"]
    exp[(a < m1) & (e > m0)] = V["MMIO"]
    exp[(a >= p1) & (e <= u1)] = V["ALLOW"]
    v, _, _ = oracle.check_batch(syn.table1_apertures(), a.astype(np.uint64), w.astype(np.uint8))
    assert (v == exp).all()


# ---------------------------------------------------------------- brute force


def _tiny_table(st, window_lo, window=192, max_ranges=6):
    """Random disjoint ranges in a small window, some abutting, some gapped."""
    k = int(st.below(max_ranges + 1, 1)[0])
    cuts = np.sort(st.below(window, 2 * k)) if k else np.array([], dtype=np.int64)
    base, size, kind = [], [], []
    for i in range(k):
        lo, hi = int(cuts[2 * i]), int(cuts[2 * i + 1])
        if st.below(3, 1)[0] == 0 and base:       # abut the previous range
            lo = base[-1] + size[-1] - window_lo
        if hi <= lo:
            continue
        base.append(window_lo + lo)
        size.append(hi - lo)
        kind.append(int(st.below(3, 1)[0]))
    ident = list(range(100, 100 + len(base)))
    return syn._ranges(base, size, kind, ident)


def _bytewise(t, window_lo, window, a, w):
    """Verdict and range from the owners of the bytes [a, a+w)."""
    if w == 0 or a + w > M64:
        return V["INVALID"], oracle.NO_RANGE
    owner = {}
    for j in range(len(t)):
        for x in range(int(t.base[j]), int(t.base[j] + t.size[j])):
            owner[x] = j
    owners = {owner.get(x, -1) for x in range(a, a + w)}
    if len(owners) == 1 and -1 not in owners:
        j = next(iter(owners))
        if t.kind[j] == 0:
            return V["ALLOW"], int(t.ident[j])
    owners.discard(-1)
    for cls, verdict in ((2, "MMIO"), (1, "PROTECTED"), (0, "STRADDLE")):
        hit = [j for j in owners if t.kind[j] == cls]
        if hit:
            j = min(hit, key=lambda j: int(t.base[j]))
            return V[verdict], int(t.ident[j])
    return V["UNMAPPED"], oracle.NO_RANGE


@pytest.mark.parametrize("window_lo", [0x1000, 2**64 - 192])
def test_bruteforce_tiny_tables(window_lo):
    st = syn.Stream(11, window_lo & 0xFFFF)
    window = 192
    for trial in range(40):
        t = _tiny_table(st, window_lo, window)
        assert oracle.table_check(t) == 0
        lo = max(window_lo - 20, 0)
        hi = min(window_lo + window + 4, M64)
        addrs, widths = [], []
        for a in range(lo, hi):
            for w in (1, 2, 3, 4, 8, 16, 17):
                addrs.append(a)
                widths.append(w)
        addrs = np.array(addrs, dtype=np.uint64)
        widths = np.array(widths, dtype=np.uint64)
        exp = [_bytewise(t, window_lo, window, int(a), int(w)) for a, w in zip(addrs, widths)]
        ev = np.array([e[0] for e in exp])
        er = np.array([e[1] for e in exp])
        v, rid = oracle.validate(t, addrs, widths)
        assert (v == ev).all() and (rid == er).all()
        # batch form: widths outside {1,2,4,8,16} are invalid
        bv, brid, log = oracle.check_batch(t, addrs, widths.astype(np.uint8), method="linear")
        sv, srid, slog = oracle.check_batch(t, addrs, widths.astype(np.uint8), method="sorted")
        legal = np.isin(widths, [1, 2, 4, 8, 16])
        assert (bv[legal] == ev[legal]).all() and (bv[~legal] == V["INVALID"]).all()
        assert (brid[legal] == er[legal]).all()
        assert (sv == bv).all() and (srid == brid).all() and slog == log
        viol = np.flatnonzero(bv != 0)
        assert log.count == len(viol)
        if len(viol):
            i = int(viol[0])
            assert (log.key, log.addr, log.width, log.verdict, log.range_id) == \
                (i, int(addrs[i]), int(widths[i]), int(bv[i]), int(brid[i]))


# ---------------------------------------------------------------- aperture rule

APERTURE_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_aperture_rule.txt")


def test_aperture_rule_table1_golden():
    rows = []
    for line in open(APERTURE_GOLDEN):
        f = line.split()
        if f and not f[0].startswith("#"):
            rows.append((int(f[1], 16), int(f[2], 0), V[f[3]], int(f[4], 16)))
    addr = np.array([r[0] for r in rows], dtype=np.uint64)
    width = np.array([r[1] for r in rows], dtype=np.uint8)
    v, rid, log = oracle.aperture_batch(syn.table1_protected(), addr, width)
    assert v.tolist() == [r[2] for r in rows]
    assert rid.tolist() == [r[3] for r in rows]
    first = next(i for i, r in enumerate(rows) if r[2] != 0)
    assert log.key == first and log.count == sum(r[2] != 0 for r in rows)


def test_aperture_workload_labels():
    """The aperture workload places each access by construction; its verdicts are its labels."""
    n = 1 << 20
    addr, width, label = syn.aperture_accesses(n)
    v, rid, log = oracle.aperture_batch(syn.table1_protected(), addr, width)
    assert (v == label).all()
    denied = int(n * 0.04) + 2 * int(n * 0.03)
    assert int((label == 0).sum()) == n - denied and log.count == denied
    assert log.key == int(np.flatnonzero(label)[0])


@pytest.mark.parametrize("window_lo", [0x1000, 2**64 - 192])
def test_aperture_rule_bruteforce(window_lo):
    """Per-byte owners again: deny iff some byte belongs to an MMIO (first) or protected
    aperture, reporting the lowest-based one; user ranges in the tiny tables are ignored."""
    st = syn.Stream(13, window_lo & 0xFFFF)
    for trial in range(40):
        t = _tiny_table(st, window_lo)
        keep = t.kind != syn.KIND_USER
        ap = syn._ranges(t.base[keep], t.size[keep], t.kind[keep], t.ident[keep])
        lo, hi = max(window_lo - 20, 0), min(window_lo + 196, M64)
        addrs = np.repeat(np.arange(lo, hi, dtype=np.uint64), 6)
        widths = np.tile(np.array([1, 2, 3, 4, 8, 16], dtype=np.uint8), hi - lo)
        owner = {}
        for j in range(len(ap)):
            for x in range(int(ap.base[j]), int(ap.base[j] + ap.size[j])):
                owner[x] = j
        v, rid, log = oracle.aperture_batch(ap, addrs, widths)
        for i, (a, w) in enumerate(zip(addrs.tolist(), widths.tolist())):
            if w not in (1, 2, 4, 8, 16) or a + w > M64:
                assert (v[i], rid[i]) == (V["INVALID"], oracle.NO_RANGE)
                continue
            hit = {owner[x] for x in range(a, a + w) if x in owner}
            want = (V["ALLOW"], oracle.NO_RANGE)
            for cls, name in ((syn.KIND_MMIO, "MMIO"), (syn.KIND_PROTECTED, "PROTECTED")):
                js = [j for j in hit if ap.kind[j] == cls]
                if js:
                    j = min(js, key=lambda j: int(ap.base[j]))
                    want = (V[name], int(ap.ident[j]))
                    break
            assert (int(v[i]), int(rid[i])) == want, (hex(a), w)
        assert log.count == int((v != 0).sum())


def test_aperture_rule_is_the_table_rule_with_user_complement():
    """With the rest of the space given to user ranges, the table rule denies exactly what
    the aperture rule denies (the batch workload's apertures, its own accesses)."""
    t = syn.batch_table()
    addr, width, label = syn.batch_accesses(t, 1 << 16)
    keep = t.kind != syn.KIND_USER
    ap = syn._ranges(t.base[keep], t.size[keep], t.kind[keep], t.ident[keep])
    order = np.argsort(ap.base)
    b, e = ap.base[order].astype(object), (ap.base[order] + ap.size[order]).astype(object)
    ub, us = [], []
    cur = 0
    for x, y in zip(b, e):
        if x > cur:
            ub.append(cur); us.append(x - cur)
        cur = y
    ub.append(cur); us.append(M64 - cur)
    full = syn._ranges(list(ap.base) + ub, list(ap.size) + us,
                       list(ap.kind) + [syn.KIND_USER] * len(ub),
                       list(ap.ident) + list(range(0x5000, 0x5000 + len(ub))))
    va, ra, la = oracle.aperture_batch(ap, addr, width)
    vt, rt, lt = oracle.check_batch(full, addr, width, method="sorted")
    deny = va != 0
    assert deny.sum() > 0 and (vt[deny] == va[deny]).all() and (rt[deny] == ra[deny]).all()
    assert (vt[~deny] == 0).all()


def test_table_rules():
    ok = syn._ranges([0, 16, 32], [16, 16, 1], [0, 0, 1], [1, 2, 3])
    assert oracle.table_check(ok) == 0                       # abutting ranges are legal
    assert oracle.table_check(syn._ranges([0, 15], [16, 4], [0, 1], [1, 2])) == 3
    assert oracle.table_check(syn._ranges([0], [0], [0], [1])) == 1
    assert oracle.table_check(syn._ranges([M64], [1], [0], [1])) == 2
    assert oracle.table_check(syn._ranges([M64 - 1], [1], [0], [1])) == 0
    assert oracle.table_check(syn._ranges([0], [1], [3], [1])) == 4


def test_abutting_allocations_straddle():
    """Two user allocations side by side stay two: an access across both is denied."""
    t = syn._ranges([0x1000, 0x1010], [16, 16], [0, 0], [7, 8])
    v, rid, _ = oracle.check_batch(t, np.array([0x100C, 0x1008, 0x1010], np.uint64),
                                   np.array([8, 8, 16], np.uint8))
    assert v.tolist() == [V["STRADDLE"], V["ALLOW"], V["ALLOW"]]
    assert rid.tolist() == [7, 7, 8]


# ---------------------------------------------------------------- generator labels


def test_batch_workload_labels_small():
    t = syn.batch_table()
    assert oracle.table_check(t) == 0
    addr, width, label = syn.batch_accesses(t, 200_000)
    n = len(addr)
    counts = np.bincount(label, minlength=6)
    assert counts[V["STRADDLE"]] == n * 3 // 100 and counts[V["UNMAPPED"]] == n * 3 // 100
    assert counts[V["PROTECTED"]] + counts[V["MMIO"]] == n * 4 // 100
    v_lin, rid_lin, log_lin = oracle.check_batch(t, addr, width, method="linear")
    assert (v_lin == label).all()
    v_s, rid_s, log_s = oracle.check_batch(t, addr, width, method="sorted")
    assert (v_s == v_lin).all() and (rid_s == rid_lin).all() and log_s == log_lin
    assert log_lin.key == int(np.flatnonzero(label != 0)[0])
    assert log_lin.count == int((label != 0).sum())


def test_batch_workload_full_size_sorted():
    """1M accesses, the sorted oracle; labels hold exactly (90/4/3/3 split)."""
    t = syn.batch_table()
    addr, width, label = syn.batch_accesses(t, 1 << 20)
    v, _, log = oracle.check_batch(t, addr, width, method="sorted")
    assert (v == label).all()
    assert log.count == (1 << 20) - int((label == 0).sum())


# ---------------------------------------------------------------- reference kernels


def _f32_neighbours(r):
    r = np.float32(r)
    return np.nextafter(r, np.float32(-np.inf)), np.nextafter(r, np.float32(np.inf))


def _is_correct_rounding(exact: Fraction, r: np.float32) -> bool:
    lo, hi = _f32_neighbours(r)
    d = abs(exact - Fraction(float(r)))
    dl = abs(exact - Fraction(float(lo)))
    dh = abs(exact - Fraction(float(hi)))
    if d < dl and d < dh:
        return True
    if d == dl or d == dh:                 # tie: even significand wins
        return (np.float32(r).view(np.uint32) & 1) == 0
    return False


def test_reference_kernels_ieee():
    st = syn.Stream(5, 1)
    n = 3000
    b = (st.uniform(n) * 2 - 1).astype(np.float32) * np.float32(2.0) ** st.below(40, n).astype(np.float32)
    c = (st.uniform(n) * 2 - 1).astype(np.float32)
    s = 3.0
    assert (oracle.stream_plain("copy", b, None).view(np.uint32) == b.view(np.uint32)).all()
    scaled = oracle.stream_plain("scale", b, None, s)
    assert (scaled == np.float32(s) * b).all()
    tri = oracle.stream_plain("triad", b, c, s)
    for i in range(n):
        exact = Fraction(float(np.float32(s))) * Fraction(float(c[i])) + Fraction(float(b[i]))
        assert _is_correct_rounding(exact, tri[i]), i


def test_stream_guard_no_violation_equals_plain():
    """Sec. V-E / Fig. 2 caption: accesses to user allocations stay on the normal path,
    so a guarded kernel with no violation computes what the unguarded one does."""
    n = 1003
    r, span, off = syn.stream_layout(n, n_decoys=20, n_prot=4, n_mmio=2, decoy_max=64 * 1024)
    base = 0x7F0000000000
    t = r.shifted(base)
    va = {k: base + v for k, v in off.items()}
    st = syn.Stream(3, 3)
    b = st.uniform(n).astype(np.float32)
    c = st.uniform(n).astype(np.float32)
    for op in ("copy", "scale", "triad"):
        for pol in ("poison", "sink", "report"):
            got, log = oracle.stream(op, t, va, b, c, np.zeros(n, np.float32), 3.0, pol)
            assert (got == oracle.stream_plain(op, b, c, 3.0)).all()
            assert log.count == 0


def test_stream_guard_poison_protected_window():
    """A protected range laid over part of b: every 16-byte (or tail 4-byte) unit that
    touches it reads 0 under poison and is logged; report keeps the data."""
    n = 4 * 64 + 3
    base = 0x10000
    va = {"b": base, "c": base + 0x10000, "a": base + 0x20000}
    prot_lo, prot_len = base + 100, 300                # bytes [100, 400) of b
    t = syn._ranges([base, base + 0x10000, base + 0x20000, prot_lo],
                    [100, 4 * n, 4 * n, prot_len], [0, 0, 0, 1], [1, 2, 3, 9])
    # b is the user range [base, base+100) plus a tail user range after the protected one
    t = t.concat(syn._ranges([prot_lo + prot_len], [4 * n - 100 - prot_len], [0], [4]))
    st = syn.Stream(4, 4)
    b = st.uniform(n).astype(np.float32) + 1
    got, log = oracle.stream("copy", t, va, b, None, np.full(n, -1, np.float32), 1.0, "poison")
    units = n // 4
    starts = np.concatenate([np.arange(units) * 16, units * 16 + np.arange(n - units * 4) * 4])
    widths = np.concatenate([np.full(units, 16), np.full(n - units * 4, 4)])
    hit = (starts < 100 + prot_len) & (starts + widths > 100)
    cross = hit & ((starts < 100) | (starts + widths > 100 + prot_len))
    elem_hit = np.concatenate([np.repeat(hit[:units], 4), hit[units:]])
    assert (got[elem_hit] == 0).all() and (got[~elem_hit] == b[~elem_hit]).all()
    assert log.count == int(hit.sum())
    assert log.addr == base + int(starts[hit][0]) and log.site == 0
    assert log.verdict == V["PROTECTED"] and log.range_id == 9
    assert cross.sum() == 1          # the unit across byte 100 touches user and protected: PROTECTED
    got_r, log_r = oracle.stream("copy", t, va, b, None, np.zeros(n, np.float32), 1.0, "report")
    assert (got_r == b).all() and log_r == log


# ---------------------------------------------------------------- irregular kernels


def _irregular_case(n=4003, stripes=16, user=64 * 1024, prot=4 * 1024, bins=1 << 12,
                    frac_bad=0.01, dist="uniform", base=0x7E0000000000):
    r, span, off = syn.irregular_layout(n, stripes, user, prot, bins)
    idx, key, bad = syn.irregular_indices(n, stripes, user, prot, bins, dist=dist,
                                          frac_bad=frac_bad, seed=5)
    arena = np.zeros(span, np.uint8)
    st = syn.Stream(6, 6)
    tvals = st.uniform((stripes * (user + prot)) // 4).astype(np.float32)
    arena[:len(tvals) * 4] = tvals.view(np.uint8)
    va = {"t": base + off["t"], "idx": base + off["idx"], "out": base + off["out"],
          "bins": base + off["bins"]}
    return r.shifted(base), arena, base, va, off, idx, key, bad, tvals


def _put(arena, off, arr):
    b = np.ascontiguousarray(arr).view(np.uint8)
    arena[off:off + len(b)] = b


@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_irregular_gather_against_fancy_indexing(dist):
    """Gather with no violation is T[idx]; with indices aimed into protected tails,
    poison gives 0.0 there, report gives the tail's contents, and the log counts them."""
    t, arena, base, va, off, idx, key, bad, tvals = _irregular_case(dist=dist)
    n = len(idx)
    _put(arena, off["idx"], idx)
    for policy in ("poison", "sink", "report"):
        a = arena.copy()
        log = oracle.irregular("gather", t, a, base, va, n, policy)
        got = a[off["out"]:off["out"] + 4 * n].view(np.float32)
        want = tvals[idx]
        if policy != "report":
            want = np.where(bad, np.float32(0), want)
        assert (got == want).all()
        assert log.count == int(bad.sum())
        first = int(va["t"] + 4 * idx[bad].min())
        assert (log.key, log.addr, log.site, log.width, log.verdict) == (first, first, 2, 4, 1)


def test_irregular_scatter_and_hist_against_numpy():
    t, arena, base, va, off, idx, key, bad, tvals = _irregular_case()
    n = len(idx)
    _put(arena, off["idx"], idx)
    a = arena.copy()
    log = oracle.irregular("scatter", t, a, base, va, n, "poison")
    T = a[:len(tvals) * 4].view(np.float32)
    want = tvals.copy()
    want[idx[~bad]] = (idx[~bad] & 0xFFFFFF).astype(np.float32)
    assert (T == want).all() and log.count == int(bad.sum())
    # histogram: the key array stands in for idx, the bins for the table
    va_h = {"t": va["bins"], "idx": va["idx"]}
    a = arena.copy()
    _put(a, off["idx"], key)
    log = oracle.irregular("hist", t, a, base, va_h, n, "poison")
    bins = a[off["bins"]:off["bins"] + 4 * (1 << 12)].view(np.uint32)
    assert (bins == np.bincount(key[~bad], minlength=1 << 12)).all()
    assert log.count == int(bad.sum())
    a = arena.copy()
    _put(a, off["idx"], key)
    oracle.irregular("hist", t, a, base, va_h, n, "report")
    tail = a[off["bins"] + 4 * (1 << 12):off["bins"] + 4 * (1 << 12) + 4096].view(np.uint32)
    assert tail.sum() == int(bad.sum())          # report lets the denied increments land


def test_irregular_denied_index_load_reads_zero():
    """A protected range laid over part of the index array: under poison those index
    loads read 0, so the elements they feed gather T[0]."""
    t, arena, base, va, off, idx, key, bad, tvals = _irregular_case(frac_bad=0)
    n = len(idx)
    _put(arena, off["idx"], idx)
    # carve [32, 96) bytes of the idx array out as protected (two 16-byte loads, units 1-2)
    ranges = [(int(b), int(s), int(k), int(i)) for b, s, k, i in zip(t.base, t.size, t.kind, t.ident)]
    ix = next(j for j, x in enumerate(ranges) if x[3] == 0x12)
    b0, s0, _, _ = ranges.pop(ix)
    ranges += [(b0, 32, 0, 0x12), (b0 + 32, 64, 1, 0x99), (b0 + 96, s0 - 96, 0, 0x98)]
    t2 = syn._ranges(*zip(*ranges))
    a = arena.copy()
    log = oracle.irregular("gather", t2, a, base, va, n, "poison")
    got = a[off["out"]:off["out"] + 4 * n].view(np.float32)
    want = tvals[idx].copy()
    want[4:12] = tvals[0]
    assert (got == want).all()
    assert log.count == 4 and (log.key, log.site, log.width, log.range_id) == (b0 + 32, 0, 16, 0x99)


def _remap_case(n=4003, half=1 << 20, base=0x7E0000000000):
    r, span, off = syn.remap_layout(n, half)
    idx, key, cls = syn.remap_indices(n, half)
    arena = np.zeros(span, np.uint8)
    st = syn.Stream(6, 7)
    arena[:2 * half] = st.uniform(half // 2).astype(np.float32).view(np.uint8)
    va = {"t": base + off["t"], "idx": base + off["idx"], "out": base + off["out"]}
    return r.shifted(base), arena, base, va, off, idx, key, cls


def test_remap_gather_moves_shadow_accesses_into_the_table():
    """REMAP_OR (Sec. V-E): a denied access whose address ORed with the mask is an allowed
    access is carried out there; otherwise it is dropped as under poison. Here the mask is
    the shadow's size, so T[e] for -half/4 <= e < 0 reads T[e + half/4]; the range at 2 half
    maps into a hole, so those elements read 0. Every denied access is still logged."""
    half = 1 << 20
    t, arena, base, va, off, idx, key, cls = _remap_case(half=half)
    n = len(idx)
    _put(arena, off["idx"], idx)
    tv = arena[half:2 * half].view(np.float32).copy()
    a = arena.copy()
    log = oracle.irregular("gather", t, a, base, va, n, "remap", remap=half)
    got = a[off["out"]:off["out"] + 4 * n].view(np.float32)
    ne = half // 4
    want = np.where(cls == 0, tv[np.clip(idx, 0, ne - 1)], np.float32(0))
    want = np.where(cls == 1, tv[np.clip(idx + ne, 0, ne - 1)], want)
    assert (cls == 1).sum() > 10 and (cls == 2).sum() > 10
    assert (got == want).all()
    assert log.count == int((cls != 0).sum())
    first = int(va["t"] + 4 * idx[cls != 0].min())
    assert (log.key, log.site, log.verdict, log.range_id) == (first, 2, 1, 0x40)
    # a zero mask leaves every denied access denied: remap equals poison
    a0, a1 = arena.copy(), arena.copy()
    l0 = oracle.irregular("gather", t, a0, base, va, n, "remap", remap=0)
    l1 = oracle.irregular("gather", t, a1, base, va, n, "poison")
    assert (a0 == a1).all() and l0 == l1


def test_aperture_rule_in_kernels_sees_only_the_apertures():
    """Under the aperture rule the gather's denials are exactly the accesses into the
    protected apertures; an access into a hole, which the table rule denies, reads the
    hole's contents."""
    half = 1 << 20
    t, arena, base, va, off, idx, key, cls = _remap_case(half=half)
    n, ne = len(idx), half // 4
    idx = idx.copy()
    hole = np.arange(0, n, 97)
    idx[hole] = 2 * ne + (np.arange(len(hole)) % 1000)   # [3 half, 3 half + 4000): a hole
    cls = cls.copy()
    cls[hole] = 3
    arena[3 * half:3 * half + 4000] = (np.arange(4000) % 251 + 1).astype(np.uint8)
    _put(arena, off["idx"], idx)
    tv = arena[half:2 * half].view(np.float32)
    hv = arena[3 * half:3 * half + 4000].view(np.float32)
    keep = t.kind != syn.KIND_USER
    ap = syn._ranges(t.base[keep], t.size[keep], t.kind[keep], t.ident[keep])
    for rule, r in (("aperture", ap), ("table", t)):
        a = arena.copy()
        log = oracle.irregular("gather", r, a, base, va, n, "poison", rule=rule)
        got = a[off["out"]:off["out"] + 4 * n].view(np.float32)
        want = np.where(cls == 0, tv[np.clip(idx, 0, ne - 1)], np.float32(0))
        if rule == "aperture":
            want = np.where(cls == 3, hv[np.clip(idx - 2 * ne, 0, 999)], want)
        assert (got == want).all(), rule
        denied = (cls == 1) | (cls == 2) | ((cls == 3) & (rule == "table"))
        assert log.count == int(denied.sum()), rule


def test_remap_scatter_and_hist():
    half = 1 << 20
    t, arena, base, va, off, idx, key, cls = _remap_case(half=half)
    n, ne = len(idx), half // 4
    _put(arena, off["idx"], idx)
    a = arena.copy()
    log = oracle.irregular("scatter", t, a, base, va, n, "remap", remap=half)
    T = arena[half:2 * half].view(np.float32).copy()
    for e, c in zip(idx, cls):                       # in order: later writes win
        if c == 0:
            T[e] = np.float32(e & 0xFFFFFF)
        elif c == 1:
            T[e + ne] = np.float32(e & 0xFFFFFF)
    assert (a[half:2 * half].view(np.float32) == T).all()
    assert (a[:half] == arena[:half]).all()          # the shadow is never written
    assert log.count == int((cls != 0).sum())
    va_h = {"t": base + off["bins"], "idx": va["idx"]}
    a = arena.copy()
    _put(a, off["idx"], key)
    log = oracle.irregular("hist", t, a, base, va_h, n, "remap", remap=half)
    bins = a[off["bins"]:off["bins"] + half].view(np.uint32)
    want = np.bincount(key[cls == 0], minlength=ne) + np.bincount(key[cls == 1] + ne, minlength=ne)
    assert (bins == want).all() and log.count == int((cls != 0).sum())


def test_dma_exact_allocation():
    """Sec. V-C: DMA registration is accepted only for an exact live user allocation."""
    t = syn._ranges([0x1000, 0x2000, 0x3000], [0x800, 0x400, 0x100], [0, 0, 1], [1, 2, 3])
    cases = [  # (ptr, bytes, verdict)
        (0x1000, 0x800, "ALLOW"), (0x2000, 0x400, "ALLOW"),
        (0x1000, 0x7FF, "NOT_EXACT"), (0x1001, 0x7FF, "NOT_EXACT"), (0x2100, 0x10, "NOT_EXACT"),
        (0x1000, 0x801, "STRADDLE"), (0x3000, 0x100, "PROTECTED"), (0x5000, 0x10, "UNMAPPED"),
        (0x1000, 0, "INVALID"),
    ]
    v, rid = oracle.validate_exact(t, np.array([c[0] for c in cases], np.uint64),
                                   np.array([c[1] for c in cases], np.uint64))
    assert [oracle.VERDICT_NAMES[x] for x in v] == [c[2] for c in cases]
    assert rid[:2].tolist() == [1, 2] and rid[2] == 1


@pytest.mark.parametrize("seed", [1, 2])
def test_dma_exact_random_against_membership(seed):
    """Exact-match membership in the set of user (base, size) pairs decides ALLOW; every
    other pair carries validate's verdict, with ALLOW turned into NOT_EXACT."""
    t = syn.batch_table(seed=syn.SEED_BASE + 70 + seed)
    st = syn.Stream(seed, 71)
    users = np.flatnonzero(t.kind == 0)
    n = 3000
    j = users[st.below(len(users), n)]
    shrink = st.below(3, n)                       # 0: exact, 1: shorter, 2: later start
    ptr = t.base[j].astype(np.int64) + np.where(shrink == 2, 256, 0)
    nb = t.size[j].astype(np.int64) - np.where(shrink > 0, 256, 0)
    v, _ = oracle.validate_exact(t, ptr.astype(np.uint64), nb.astype(np.uint64))
    exact = set(zip(t.base[users].tolist(), t.size[users].tolist()))
    want_allow = np.array([(int(p), int(b)) in exact for p, b in zip(ptr, nb)])
    assert ((v == 0) == want_allow).all()
    assert (v[~want_allow] == 6).all()            # all are inside an allocation
