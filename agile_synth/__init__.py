"""Seeded synthetic inputs for the kernel memory guard.

This module only *places* things: guard-table ranges laid out in a virtual-address
window, and access streams aimed at chosen places in that layout, each access carrying
the class it was aimed at (its label). It computes no guard verdict: the classification
rule of the protected memory model (Sec. IV-E, Sec. V-C) lives in the oracle and in the
CUDA library, and neither is imported here. Both sides consume these inputs.

Randomness is a counter-based stream: word i of stream (seed, tag) is
splitmix64(key ^ (i * 0x9E3779B97F4A7C15)) with key = splitmix64(seed ^ tag * C),
where splitmix64 is the finaliser of Steele, Lea and Flood, "Fast splittable
pseudorandom number generators" (OOPSLA 2014). Zipf draws use the rejection-inversion
method of Hoermann and Derflinger, "Rejection-inversion to generate variates from
monotone discrete distributions" (ACM TOMACS 1996), in float64 on the host.

Kinds: 0 = user allocation, 1 = protected kernel/module memory, 2 = MMIO aperture
(Table I). Labels use the verdict codes 0 = allow, 1 = protected, 2 = MMIO,
3 = straddle, 4 = unmapped, 5 = invalid.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

U64 = np.uint64
GOLDEN = U64(0x9E3779B97F4A7C15)

KIND_USER, KIND_PROTECTED, KIND_MMIO = 0, 1, 2
LABEL_ALLOW, LABEL_PROTECTED, LABEL_MMIO, LABEL_STRADDLE, LABEL_UNMAPPED, LABEL_INVALID = range(6)

# Table I of the paper: the prototype's fixed virtual-address apertures.
TABLE1_MMIO = (0xF0000000000, 0xF1000000000)
TABLE1_PROTECTED = (0xF1000000000, 0xF8000000000)
TABLE1_USER = (0xF8000000000, 0x108000000000)

SEED_BASE = 0xA61E0500
WIDTHS = np.array([1, 2, 4, 8, 16], dtype=np.uint8)

KiB = 1 << 10
MiB = 1 << 20
GiB = 1 << 30


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(x, dtype=U64) + GOLDEN
    z = (z ^ (z >> U64(30))) * U64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> U64(27))) * U64(0x94D049BB133111EB)
    return z ^ (z >> U64(31))


class Stream:
    """Counter-based random stream; every draw advances the counter by its length."""

    def __init__(self, seed: int, tag: int = 0):
        mix = np.array([(seed ^ (tag * 0x2545F4914F6CDD1D)) & (2**64 - 1)], dtype=U64)
        self.key = splitmix64(mix)[0]
        self.ctr = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.ctr, self.ctr + n, dtype=U64)
        self.ctr += n
        return splitmix64(self.key ^ (idx * GOLDEN))

    def uniform(self, n: int) -> np.ndarray:
        """float64 in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> U64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def below(self, hi, n: int) -> np.ndarray:
        """Integers in [0, hi) (hi scalar or array, each < 2**53), as int64."""
        hi = np.asarray(hi, dtype=np.float64)
        r = np.floor(self.uniform(n) * hi).astype(np.int64)
        return np.minimum(r, np.asarray(hi, dtype=np.int64) - 1)

    def log_uniform(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers log-uniform in [lo, hi]."""
        u = self.uniform(n)
        v = np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
        return np.clip(v, lo, hi)

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.u64(n), kind="stable")

    def choice(self, options: np.ndarray, n: int) -> np.ndarray:
        return options[self.below(len(options), n)]


def zipf(stream: Stream, s: float, n_max: int, count: int) -> np.ndarray:
    """Zipf(s) ranks in [1, n_max] by rejection-inversion (Hoermann & Derflinger 1996).

    The hat is the integral of x**-s; a candidate k is accepted when it falls in the
    region under the step function h(k) = k**-s. Valid for s > 1.
    """
    one_m_s = 1.0 - s

    def H(x):
        return np.power(x, one_m_s) / one_m_s

    def H_inv(y):
        return np.power(y * one_m_s, 1.0 / one_m_s)

    h_x1 = H(1.5) - 1.0
    h_n = H(n_max + 0.5)
    squeeze = 2.0 - H_inv(H(2.5) - 2.0 ** (-s))
    out = np.empty(count, dtype=np.int64)
    todo = np.arange(count)
    while todo.size:
        u = h_n + stream.uniform(todo.size) * (h_x1 - h_n)
        x = H_inv(u)
        k = np.clip(np.floor(x + 0.5), 1, n_max)
        ok = (k - x <= squeeze) | (u >= H(k + 0.5) - np.power(k, -s))
        out[todo[ok]] = k[ok].astype(np.int64)
        todo = todo[~ok]
    return out


@dataclass
class Ranges:
    """A guard table as the caller hands it over: parallel arrays, any order."""

    base: np.ndarray  # uint64
    size: np.ndarray  # uint64
    kind: np.ndarray  # uint32
    ident: np.ndarray  # uint32, caller tag reported in violation records
    meta: dict = field(default_factory=dict)

    def __len__(self):
        return len(self.base)

    def shifted(self, delta: int) -> "Ranges":
        return Ranges(self.base + U64(delta), self.size.copy(), self.kind.copy(),
                      self.ident.copy(), dict(self.meta))

    def concat(self, other: "Ranges") -> "Ranges":
        return Ranges(np.concatenate([self.base, other.base]),
                      np.concatenate([self.size, other.size]),
                      np.concatenate([self.kind, other.kind]),
                      np.concatenate([self.ident, other.ident]), dict(self.meta))


def _ranges(base, size, kind, ident, **meta) -> Ranges:
    return Ranges(np.asarray(base, dtype=U64), np.asarray(size, dtype=U64),
                  np.asarray(kind, dtype=np.uint32), np.asarray(ident, dtype=np.uint32), meta)


def table1_apertures() -> Ranges:
    """Table I as a three-range table: MMIO, protected and user apertures."""
    spans = [TABLE1_MMIO, TABLE1_PROTECTED, TABLE1_USER]
    return _ranges([s[0] for s in spans], [s[1] - s[0] for s in spans],
                   [KIND_MMIO, KIND_PROTECTED, KIND_USER], [2, 1, 0])


def table1_protected() -> Ranges:
    """Table I's two protected apertures (MMIO, then kernel/module memory): the aperture
    set of the aperture-only rule."""
    (m0, m1), (p0, p1) = TABLE1_MMIO, TABLE1_PROTECTED
    return _ranges([m0, p0], [m1 - m0, p1 - p0], [KIND_MMIO, KIND_PROTECTED], [2, 1])


def aperture_accesses(n: int, seed: int = SEED_BASE + 7):
    """(address, width, label) against Table I's protected apertures: 90% inside the user
    aperture, 4% inside the kernel/module aperture, 3% inside the MMIO aperture and 3%
    across an aperture edge (the lower MMIO edge and the MMIO/protected edge, labelled
    MMIO; the protected/user edge, labelled PROTECTED; equal thirds). Shuffled."""
    st = Stream(seed, 11)
    n_p, n_m, n_e = int(n * 0.04), int(n * 0.03), int(n * 0.03)
    n_ok = n - n_p - n_m - n_e
    parts = []
    for cnt, (lo, hi), lab in ((n_ok, TABLE1_USER, LABEL_ALLOW), (n_p, TABLE1_PROTECTED, LABEL_PROTECTED),
                               (n_m, TABLE1_MMIO, LABEL_MMIO)):
        w = st.choice(WIDTHS, cnt).astype(np.int64)
        parts.append((lo + st.below(hi - lo - w + 1, cnt), w, np.full(cnt, lab, np.uint8)))
    w = st.choice(WIDTHS[1:], n_e).astype(np.int64)
    k = 1 + st.below(w - 1, n_e)
    which = st.below(3, n_e)
    edge = np.array([TABLE1_MMIO[0], TABLE1_MMIO[1], TABLE1_PROTECTED[1]], dtype=np.int64)[which]
    lab = np.where(which == 2, LABEL_PROTECTED, LABEL_MMIO).astype(np.uint8)
    parts.append((edge - k, w, lab))
    addr = np.concatenate([p[0] for p in parts])
    width = np.concatenate([p[1] for p in parts]).astype(np.uint8)
    label = np.concatenate([p[2] for p in parts])
    p = st.permutation(n)
    return addr[p].astype(U64), width[p], label[p]


def _round_up(x, m):
    return (x + m - 1) // m * m


def layout(stream: Stream, sizes: np.ndarray, kinds: np.ndarray, span: int, base: int,
           min_gap: int = 4 * KiB, align: int = 256) -> Ranges:
    """Place ranges of the given sizes/kinds in shuffled order inside [base, base+span).

    Each range starts on an `align` boundary, its size is kept exact (not rounded), and
    every range is preceded and followed by a hole of at least `min_gap` bytes; the
    leftover span is split at random among the holes. Range i of the input gets ident
    0x1000 + i. The result is returned in an order that differs from address order.
    """
    n = len(sizes)
    sizes = np.asarray(sizes, dtype=np.int64)
    kinds = np.asarray(kinds)
    order = stream.permutation(n)          # address order -> input index
    footprint = int(_round_up(sizes, align).sum())
    holes = n + 1
    units = (span - footprint) // align
    min_units = min_gap // align
    extra = units - holes * min_units
    if extra < 0:
        raise ValueError("span too small for the requested ranges")
    w = stream.uniform(holes) + 1e-9
    share = np.floor(w / w.sum() * extra).astype(np.int64)
    share[-1] += extra - share.sum()
    gap = (share + min_units) * align
    starts = np.empty(n, dtype=np.int64)
    cur = base + int(gap[0])
    for slot in range(n):
        i = order[slot]
        starts[i] = cur
        cur += int(_round_up(int(sizes[i]), align)) + int(gap[slot + 1])
    shuffle = stream.permutation(n)        # output position -> input index
    return _ranges(starts[shuffle], sizes[shuffle], kinds[shuffle], 0x1000 + shuffle,
                   span_lo=base, span_hi=base + span)


def find(r: Ranges, ident: int) -> int:
    """Base address of the range carrying `ident`."""
    return int(r.base[np.flatnonzero(r.ident == ident)[0]])


def batch_table(seed: int = SEED_BASE + 1, span: int = GiB, base: int = TABLE1_USER[0],
                n_user: int = 64, n_prot: int = 16, n_mmio: int = 4) -> Ranges:
    """The batch-check table: 64 user (4 KiB-8 MiB), 16 protected (64 KiB-1 MiB) and
    4 MMIO (4 KiB-64 KiB) ranges in a 1 GiB window starting at the user aperture."""
    st = Stream(seed, 1)
    sizes = np.concatenate([st.log_uniform(4 * KiB, 8 * MiB, n_user),
                            st.log_uniform(64 * KiB, MiB, n_prot),
                            st.log_uniform(4 * KiB, 64 * KiB, n_mmio)])
    kinds = np.array([KIND_USER] * n_user + [KIND_PROTECTED] * n_prot + [KIND_MMIO] * n_mmio)
    return layout(st, sizes, kinds, span, base)


def _sorted(r: Ranges):
    o = np.argsort(r.base, kind="stable")
    return r.base[o].astype(np.int64), r.size[o].astype(np.int64), r.kind[o]


def batch_accesses(table: Ranges, n: int, seed: int = SEED_BASE + 1,
                   frac_deny_in=0.04, frac_straddle=0.03, frac_unmapped=0.03):
    """(address, width, label) triples aimed at the table: inside user allocations,
    inside protected/MMIO ranges, straddling a user allocation's first or last byte into
    its neighbouring hole, and inside holes or outside the window. Shuffled.

    Relies on the layout() property that every range is surrounded by holes of at least
    4 KiB, so a straddle touches exactly one range and a hole access touches none.
    """
    st = Stream(seed, 2)
    base, size, kind = _sorted(table)
    end = base + size
    n_in = int(n * frac_deny_in)
    n_str = int(n * frac_straddle)
    n_un = int(n * frac_unmapped)
    n_ok = n - n_in - n_str - n_un
    addr = np.empty(n, dtype=np.int64)
    width = np.empty(n, dtype=np.uint8)
    label = np.empty(n, dtype=np.uint8)
    users = np.flatnonzero(kind == KIND_USER)
    denies = np.flatnonzero(kind != KIND_USER)
    pos = 0

    # inside one user allocation
    w = st.choice(WIDTHS, n_ok).astype(np.int64)
    j = users[st.below(len(users), n_ok)]
    off = st.below(size[j] - w + 1, n_ok)
    addr[pos:pos + n_ok], width[pos:pos + n_ok], label[pos:pos + n_ok] = base[j] + off, w, LABEL_ALLOW
    pos += n_ok

    # inside a protected or MMIO range
    if n_in:
        w = st.choice(WIDTHS, n_in).astype(np.int64)
        j = denies[st.below(len(denies), n_in)]
        off = st.below(size[j] - w + 1, n_in)
        addr[pos:pos + n_in], width[pos:pos + n_in] = base[j] + off, w
        label[pos:pos + n_in] = np.where(kind[j] == KIND_MMIO, LABEL_MMIO, LABEL_PROTECTED)
        pos += n_in

    # straddling the first or last byte of a user allocation
    if n_str:
        w = st.choice(WIDTHS[1:], n_str).astype(np.int64)
        j = users[st.below(len(users), n_str)]
        k = 1 + st.below(w - 1, n_str)
        at_end = st.below(2, n_str) == 1
        addr[pos:pos + n_str] = np.where(at_end, end[j] - k, base[j] - k)
        width[pos:pos + n_str], label[pos:pos + n_str] = w, LABEL_STRADDLE
        pos += n_str

    # in a hole between ranges, or outside the window
    if n_un:
        w = st.choice(WIDTHS, n_un).astype(np.int64)
        lo = np.concatenate([[table.meta["span_lo"]], end])
        hi = np.concatenate([base, [table.meta["span_hi"]]])
        g = st.below(len(lo), n_un)
        in_hole = st.below(2, n_un) == 0
        a_hole = lo[g] + st.below(hi[g] - lo[g] - w + 1, n_un)
        below = st.below(2, n_un) == 0
        far = st.below(GiB, n_un)
        a_out = np.where(below, table.meta["span_lo"] - GiB + far - 16,
                         table.meta["span_hi"] + far)
        addr[pos:pos + n_un] = np.where(in_hole, a_hole, a_out)
        width[pos:pos + n_un], label[pos:pos + n_un] = w, LABEL_UNMAPPED
        pos += n_un

    p = st.permutation(n)
    return addr[p].astype(U64), width[p], label[p]


def stream_layout(n_elems: int, seed: int = SEED_BASE + 2, n_decoys: int = 1021,
                  n_prot: int = 64, n_mmio: int = 8, decoy_max: int = 8 * MiB):
    """Arena layout for the guarded streaming kernels: three fp32 arrays a, b, c of
    n_elems each plus decoy user allocations, protected and MMIO ranges, all carved
    from one arena the caller owns. Offsets are relative to the arena start.

    Returns (ranges_relative, arena_bytes, {"a": off, "b": off, "c": off}).
    """
    st = Stream(seed, 3)
    arr = n_elems * 4
    sizes = np.concatenate([[arr, arr, arr],
                            st.log_uniform(4 * KiB, decoy_max, n_decoys),
                            st.log_uniform(64 * KiB, MiB, n_prot),
                            st.log_uniform(4 * KiB, 64 * KiB, n_mmio)])
    kinds = np.array([KIND_USER] * (3 + n_decoys) + [KIND_PROTECTED] * n_prot
                     + [KIND_MMIO] * n_mmio)
    align = 4 * KiB
    holes = len(sizes) + 1
    need = int(_round_up(sizes, align).sum()) + holes * 64 * KiB
    span = _round_up(need, 2 * MiB)
    r = layout(st, sizes, kinds, span, 0, min_gap=4 * KiB, align=align)
    return r, span, {name: find(r, 0x1000 + k) for k, name in enumerate("abc")}


# ---------------------------------------------------------------- irregular access

ODD_MIX = 0x9E3779B1          # odd: multiplication by it permutes residues mod 2^k


def irregular_layout(n_idx: int, stripes: int = 4096, user_bytes: int = 4 * MiB,
                     prot_bytes: int = 64 * KiB, bins: int = 1 << 20):
    """Arena layout for gather / scatter / histogram: a table region of `stripes` user
    allocations of `user_bytes`, each followed by a protected range of `prot_bytes`
    (protected ranges interleaved through the table); a bins array (u32) followed by a
    protected range; the int64 index array and the fp32 output array. Offsets are relative
    to the arena start; all arrays are 256-byte aligned.

    Returns (ranges_relative, arena_bytes, offsets {'t', 'bins', 'idx', 'out'}).
    """
    stripe = user_bytes + prot_bytes
    base, size, kind, ident = [], [], [], []
    for s in range(stripes):
        base += [s * stripe, s * stripe + user_bytes]
        size += [user_bytes, prot_bytes]
        kind += [KIND_USER, KIND_PROTECTED]
        ident += [0x20000 + s, 0x30000 + s]
    cur = stripes * stripe + 64 * KiB
    off = {"t": 0, "bins": cur}
    base += [cur, cur + 4 * bins]
    size += [4 * bins, prot_bytes]
    kind += [KIND_USER, KIND_PROTECTED]
    ident += [0x10, 0x11]
    cur = _round_up(cur + 4 * bins + prot_bytes + 64 * KiB, 256)
    off["idx"] = cur
    base.append(cur); size.append(8 * n_idx); kind.append(KIND_USER); ident.append(0x12)
    cur = _round_up(cur + 8 * n_idx + 64 * KiB, 256)
    off["out"] = cur
    base.append(cur); size.append(4 * n_idx); kind.append(KIND_USER); ident.append(0x13)
    cur = _round_up(cur + 4 * n_idx + 64 * KiB, 2 * MiB)
    return _ranges(base, size, kind, ident, stripes=stripes, user_bytes=user_bytes,
                   prot_bytes=prot_bytes, bins=bins), cur, off


def irregular_indices(n: int, stripes: int = 4096, user_bytes: int = 4 * MiB,
                      prot_bytes: int = 64 * KiB, bins: int = 1 << 20, dist: str = "uniform",
                      frac_bad: float = 0.001, seed: int = SEED_BASE + 3, chunk: int = 1 << 24):
    """int64 element offsets into the table region and histogram keys into the bins.

    A rank r is drawn over the user elements (uniform, or Zipf(1.1) with the rank mixed
    by an odd multiplier modulo the user element count, a power of two, so hot elements
    are spread over the table) and mapped to its stripe and position. Exactly
    int(n * frac_bad) accesses, at random positions, are aimed into protected ranges
    instead: a table index into a stripe's protected tail, and a key into the protected
    range after the bins. Returns (idx, key, bad) with bad marking those positions.
    """
    st = Stream(seed, 9)
    ue = user_bytes // 4
    se = (user_bytes + prot_bytes) // 4
    pe = prot_bytes // 4
    total = stripes * ue
    idx = np.empty(n, dtype=np.int64)
    key = np.empty(n, dtype=np.int64)
    for lo in range(0, n, chunk):
        m = min(chunk, n - lo)
        if dist == "uniform":
            r = st.below(total, m)
        elif dist == "zipf":
            assert total & (total - 1) == 0, "Zipf mixing needs a power-of-two element count"
            k = zipf(st, 1.1, total, m) - 1
            r = ((k.astype(np.uint64) * U64(ODD_MIX)) & U64(total - 1)).astype(np.int64)
        else:
            raise ValueError(dist)
        idx[lo:lo + m] = (r // ue) * se + r % ue
        key[lo:lo + m] = r & (bins - 1)
    nbad = int(n * frac_bad)
    bad = np.zeros(n, dtype=bool)
    if nbad:
        pos = np.unique(st.below(n, nbad))
        while len(pos) < nbad:                  # redraw the few collisions
            pos = np.unique(np.concatenate([pos, st.below(n, nbad - len(pos))]))
        bad[pos] = True
        s_ = st.below(stripes, len(pos))
        idx[pos] = s_ * se + ue + st.below(pe, len(pos))
        key[pos] = bins + st.below(pe, len(pos))
    return idx, key, bad


def remap_layout(n_idx: int, half: int = MiB):
    """Arena layout for the REMAP_OR policy with mask `half` (a power of two); the arena
    start must be aligned to 2 * half. Block [0, 2 half): a protected shadow in the lower
    half under the user table T in the upper half, so an access into the shadow ORed with
    the mask lands in T. Then a protected range at 2 half whose ORed image, 3 half on, is a
    hole; a second shadow/user pair at [4 half, 6 half) holding the bins (half / 4 u32);
    the int64 index array and the fp32 output array.

    Returns (ranges_relative, arena_bytes, offsets {'t', 'bins', 'idx', 'out'}).
    """
    assert half & (half - 1) == 0 and half >= 64 * KiB
    base = [0, half, 2 * half, 4 * half, 5 * half]
    size = [half, half, 64 * KiB, half, half]
    kind = [KIND_PROTECTED, KIND_USER, KIND_PROTECTED, KIND_PROTECTED, KIND_USER]
    ident = [0x40, 0x41, 0x42, 0x43, 0x10]
    off = {"t": half, "bins": 5 * half, "idx": 6 * half + 64 * KiB}
    base.append(off["idx"]); size.append(8 * n_idx); kind.append(KIND_USER); ident.append(0x12)
    off["out"] = _round_up(off["idx"] + 8 * n_idx + 64 * KiB, 256)
    base.append(off["out"]); size.append(4 * n_idx); kind.append(KIND_USER); ident.append(0x13)
    span = _round_up(off["out"] + 4 * n_idx + 64 * KiB, 2 * half)
    return _ranges(base, size, kind, ident, half=half), span, off


def remap_indices(n: int, half: int = MiB, frac_bad: float = 0.02, seed: int = SEED_BASE + 6):
    """Element offsets for remap_layout: uniform over T (and over the bins for the keys).
    int(n * frac_bad) positions are aimed off the buffer: alternately into the shadow below
    it (negative offsets; class 1) and into the protected range at 2 half (class 2).
    Returns (idx, key, cls) with cls 0 for an in-buffer access."""
    st = Stream(seed, 10)
    ne = half // 4
    idx = st.below(ne, n).astype(np.int64)
    key = st.below(ne, n).astype(np.int64)
    cls = np.zeros(n, dtype=np.int8)
    nbad = int(n * frac_bad)
    if nbad:
        pos = np.unique(st.below(n, nbad))
        c = np.where(np.arange(len(pos)) % 2 == 0, 1, 2).astype(np.int8)
        cls[pos] = c
        j = st.below(16 * KiB, len(pos)).astype(np.int64)
        sh = -1 - st.below(ne, len(pos)).astype(np.int64)
        # T starts at half: the shadow is [-ne, 0), the range at 2 half is ne + j;
        # the bins start at 5 half: the shadow is [-ne, 0), the range at 2 half is -3 ne + j
        idx[pos] = np.where(c == 1, sh, ne + j)
        key[pos] = np.where(c == 1, sh, -3 * ne + j)
    return idx, key, cls


# ---------------------------------------------------------------- many clients

def lognormal(stream: Stream, median: float, sigma: float, n: int) -> np.ndarray:
    """Lognormal draws (Box-Muller normals, float64)."""
    u1 = stream.uniform(n) * (1 - 1e-12) + 1e-12
    u2 = stream.uniform(n)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2 * np.pi * u2)
    return median * np.exp(sigma * z)


def client_specs(n_clients: int = 256, seed: int = SEED_BASE + 4, median: int = 2 * MiB,
                 sigma: float = float(np.log(128) / 3), lo: int = 4 * KiB, hi: int = 256 * MiB,
                 table_lo: int = 8, table_hi: int = 4096, mix=(0.5, 0.3, 0.2)):
    """Per-client kernel kind (copy / gather / hist in the given mix), buffer size
    (lognormal, clamped to [lo, hi], 256-byte multiple) and table size (log-uniform)."""
    st = Stream(seed, 11)
    counts = [int(round(m * n_clients)) for m in mix]
    counts[0] += n_clients - sum(counts)
    ops = np.array(["copy"] * counts[0] + ["gather"] * counts[1] + ["hist"] * counts[2])
    ops = ops[st.permutation(n_clients)]
    size = np.clip(lognormal(st, median, sigma, n_clients), lo, hi).astype(np.int64) // 256 * 256
    ranges = st.log_uniform(table_lo, table_hi, n_clients)
    return [{"client": i, "op": str(ops[i]), "bytes": int(size[i]), "ranges": int(ranges[i])}
            for i in range(n_clients)]


HIST_BINS = 1 << 14


def client_buffers(spec: dict):
    """Buffers a client's kernel uses: name -> bytes, and its element count n."""
    B = spec["bytes"]
    if spec["op"] == "copy":
        return {"a": B, "b": B}, B // 4
    if spec["op"] == "gather":
        n = max(B // 16, 1)
        return {"t": B, "idx": 8 * n, "out": 4 * n}, n
    n = max(B // 8, 1)
    return {"bins": 4 * HIST_BINS, "idx": 8 * n}, n


def client_layout(spec: dict, seed: int = SEED_BASE + 4):
    """A client's arena: its buffers as user allocations plus decoy allocations (user,
    protected, MMIO; 4-64 KiB) up to its table size, every range surrounded by holes.
    Returns (ranges_relative, arena_bytes, {buffer: offset}, n)."""
    st = Stream(seed, 100 + spec["client"])
    bufs, n = client_buffers(spec)
    names = list(bufs)
    nd = max(spec["ranges"] - len(names), 0)
    dsize = st.log_uniform(4 * KiB, 64 * KiB, nd)
    u = st.uniform(nd)
    dkind = np.where(u < 0.9, KIND_USER, np.where(u < 0.98, KIND_PROTECTED, KIND_MMIO))
    sizes = np.concatenate([[bufs[k] for k in names], dsize]).astype(np.int64)
    kinds = np.concatenate([[KIND_USER] * len(names), dkind])
    span = _round_up(int(_round_up(sizes, 256).sum()) + (len(sizes) + 1) * 8 * KiB, 2 * MiB)
    r = layout(st, sizes, kinds, span, 0, min_gap=4 * KiB, align=256)
    return r, span, {k: find(r, 0x1000 + i) for i, k in enumerate(names)}, n


def client_indices(spec: dict, n: int, seed: int = SEED_BASE + 4, frac_bad: float = 0.0,
                   bad_target: int | None = None):
    """Gather offsets (uniform over the table's elements) or histogram keys (uniform over
    the bins); int(n * frac_bad) of them, at random positions, are replaced by the element
    offset `bad_target` (an address the caller picked outside the client's user ranges)."""
    st = Stream(seed, 200 + spec["client"])
    hi = spec["bytes"] // 4 if spec["op"] == "gather" else HIST_BINS
    idx = st.below(hi, n)
    nbad = int(n * frac_bad)
    if nbad and bad_target is not None:
        idx[np.unique(st.below(n, nbad))] = bad_target
    return idx


# ---------------------------------------------------------------- serving

SERVE_SLOTS = 4


def serve_specs(n_clients: int = 64, seed: int = SEED_BASE + 5, median: int = 8 * MiB,
                lo: int = 64 * KiB, hi: int = 1 * GiB, **kw):
    """64 clients in the batched mix, one buffer size each (lognormal, median 8 MiB,
    clamped to [64 KiB, 1 GiB])."""
    return client_specs(n_clients, seed=seed, median=median, lo=lo, hi=hi, table_lo=8,
                        table_hi=512, **kw)


def serve_layout(spec: dict, seed: int = SEED_BASE + 5, slots: int = SERVE_SLOTS):
    """A served client's arena: its input buffers, `slots` output buffers (requests of a
    client take turns on them), decoys, and four decoy allocations that are later freed
    (kept out of the table). Returns (ranges_relative, freed_mask, arena_bytes,
    {buffer: offset}, {buffer: bytes}, n)."""
    st = Stream(seed, 300 + spec["client"])
    B = spec["bytes"]
    if spec["op"] == "copy":
        n = B // 4
        bufs = {"b": B} | {f"out{k}": B for k in range(slots)}
    elif spec["op"] == "gather":
        n = max(B // 16, 1)
        bufs = {"t": B, "idx": 8 * n} | {f"out{k}": 4 * n for k in range(slots)}
    else:
        n = max(B // 8, 1)
        bufs = {"idx": 8 * n} | {f"out{k}": 4 * HIST_BINS for k in range(slots)}
    names = list(bufs)
    nd = max(spec["ranges"] - len(names), 8)
    dsize = st.log_uniform(4 * KiB, 64 * KiB, nd)
    u = st.uniform(nd)
    dkind = np.where(u < 0.8, KIND_USER, np.where(u < 0.95, KIND_PROTECTED, KIND_MMIO))
    dkind[:2] = KIND_PROTECTED                       # every client has protected decoys
    sizes = np.concatenate([[bufs[k] for k in names], dsize]).astype(np.int64)
    kinds = np.concatenate([[KIND_USER] * len(names), dkind])
    freed_ids = set(range(0x1000 + len(names) + 2, 0x1000 + len(names) + 6))
    span = _round_up(int(_round_up(sizes, 256).sum()) + (len(sizes) + 1) * 8 * KiB, 2 * MiB)
    r = layout(st, sizes, kinds, span, 0, min_gap=4 * KiB, align=256)
    freed = np.isin(r.ident, list(freed_ids)) & (r.kind == KIND_USER)
    return r, freed, span, {k: find(r, 0x1000 + i) for i, k in enumerate(names)}, bufs, n


def poisson_arrivals(stream: Stream, rate: float, n: int) -> np.ndarray:
    """Arrival times (ns) of a Poisson process of `rate` per second."""
    gaps = -np.log(1.0 - stream.uniform(n)) / rate
    return (np.cumsum(gaps) * 1e9).astype(np.int64)


def serve_requests(layouts, rate: float, n: int, seed: int = SEED_BASE + 5,
                   frac_bad: float = 0.005, start_ns: int = 0):
    """Requests from the clients: Poisson arrivals at `rate`, a uniformly chosen client,
    its next output slot in turn, 1-16 pointer arguments (the buffers the kernel touches,
    then sub-ranges of the client's buffers), and for int(n * frac_bad) of them one
    argument replaced by a bad pointer -- into a protected decoy, into a freed allocation,
    or straddling the end of a buffer, in equal thirds. Offsets are arena-relative.

    Returns a list of dicts: client, slot, arrival_ns, args [(off, bytes)], bad (None or
    'protected' / 'freed' / 'straddle'), bad_arg."""
    st = Stream(seed, 400 + int(rate))
    arr = poisson_arrivals(st, rate, n) + start_ns
    who = st.below(len(layouts), n)
    nargs = 1 + st.below(16, n)
    nbad = int(n * frac_bad)
    bad_pos = set(np.unique(st.below(n, nbad)).tolist()) if nbad else set()
    turn = [0] * len(layouts)
    out = []
    for i in range(n):
        c = int(who[i])
        r, freed, span, off, sizes, _ = layouts[c]
        slot = turn[c] % SERVE_SLOTS
        turn[c] += 1
        ins = [k for k in off if not k.startswith("out")]
        touched = ins + [f"out{slot}"]
        args = [(off[k], sizes[k]) for k in touched]
        while len(args) < nargs[i]:
            k = ins[int(st.below(len(ins), 1)[0])]
            lo = int(st.below(sizes[k], 1)[0])
            ln = 1 + int(st.below(sizes[k] - lo, 1)[0])
            args.append((off[k] + lo, ln))
        args = args[:max(int(nargs[i]), len(touched))][:16]
        req = {"client": c, "slot": slot, "arrival_ns": int(arr[i]), "args": args, "bad": None,
               "bad_arg": None}
        if i in bad_pos:
            kind = ("protected", "freed", "straddle")[i % 3]
            j = int(st.below(len(args), 1)[0])
            if kind == "protected":
                p = np.flatnonzero(r.kind == KIND_PROTECTED)[0]
                args[j] = (int(r.base[p]), 16)
            elif kind == "freed":
                p = np.flatnonzero(freed)[0]
                args[j] = (int(r.base[p]), 64)
            else:
                k = touched[0]
                args[j] = (off[k] + sizes[k] - 8, 16)
            req.update(bad=kind, bad_arg=j)
        out.append(req)
    return out


def zipf_torch(generator, s: float, n_max: int, count: int, device):
    """Zipf(s) ranks in [1, n_max] by the same rejection-inversion method as `zipf`, drawn
    on a device with torch (float64), for index arrays too large to draw on the host. The
    stream comes from the torch generator, so the values differ from `zipf`'s."""
    import torch
    one_m_s = 1.0 - s

    def H(x):
        return torch.pow(x, one_m_s) / one_m_s

    def H_inv(y):
        return torch.pow(y * one_m_s, 1.0 / one_m_s)

    t = lambda v: torch.tensor(v, dtype=torch.float64, device=device)
    h_x1 = H(t(1.5)) - 1.0
    h_n = H(t(n_max + 0.5))
    squeeze = 2.0 - H_inv(H(t(2.5)) - 2.0 ** (-s))
    out = torch.empty(count, dtype=torch.int64, device=device)
    todo = torch.arange(count, device=device)
    while todo.numel():
        u = h_n + torch.rand(todo.numel(), dtype=torch.float64, generator=generator,
                             device=device) * (h_x1 - h_n)
        x = H_inv(u)
        k = torch.clamp(torch.floor(x + 0.5), 1, n_max)
        ok = (k - x <= squeeze) | (u >= H(k + 0.5) - torch.pow(k, -s))
        out[todo[ok]] = k[ok].to(torch.int64)
        todo = todo[~ok]
    return out
