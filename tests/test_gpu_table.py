"""The uploaded table image: the all-user block bitmap against a per-block brute force
over the ranges (a block's bit is set exactly when the block lies inside one user range),
for several layouts and page sizes."""
import numpy as np
import pytest
import torch

import agile_synth as syn
from gpu_util import DEV, device_table

pytestmark = pytest.mark.gpu


def brute_bits(r, lo, lg, nblocks):
    B = 1 << lg
    want = np.zeros(nblocks + 1, dtype=bool)
    for b, s, k in zip(r.base.tolist(), r.size.tolist(), r.kind.tolist()):
        if k != syn.KIND_USER:
            continue
        for blk in range(max(0, -(-(b - lo) // B)), min(nblocks, (b + s - lo) // B)):
            # block [lo + blk B, lo + (blk + 1) B) inside [b, b + s)
            assert lo + blk * B >= b and lo + (blk + 1) * B <= b + s
            want[blk] = True
    return want


def layouts():
    yield "table1", syn.table1_apertures()
    yield "batch", syn.batch_table()
    r, span, off = syn.irregular_layout(1000, stripes=64, user_bytes=(4 << 20) - 4096,
                                        prot_bytes=4096 + 100)
    yield "irregular_ragged", r.shifted(0x7E0000000000)
    r, span, off = syn.remap_layout(1000)
    yield "remap", r.shifted(0x7E0000000000)


@pytest.mark.parametrize("log2_page", [12, 16, 21])
def test_ubits_match_bruteforce(log2_page):
    for name, r in layouts():
        t, dev = device_table(r, log2_page)
        v = dev.view
        img = dev.buf.cpu().numpy()
        off = v.ubits - dev.address
        words = img[off:off + 4 * ((v.ubits_n + 1 + 31) // 32)].view(np.uint32)
        got = ((words[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(bool).ravel()
        assert (1 << v.ubits_log2) >= 4096 and v.ubits_n <= 1 << 18, name
        want = brute_bits(r, v.lo, v.ubits_log2, v.ubits_n)
        assert (got[:v.ubits_n + 1] == want).all(), name
        assert not got[v.ubits_n:].any(), name



def block_classes(r, lo, lg, nblocks):
    """Class of each block from the sorted ranges: 1 inside one user range, 3 inside one
    protected range, 2 touched by no range, 0 otherwise and for the block that ends at
    2^64; the entry past the last block is 2. Offsets are taken from lo in uint64."""
    o = np.argsort(r.base)
    rb = (r.base[o] - np.uint64(lo)).astype(np.uint64)
    re = rb + r.size[o].astype(np.uint64)
    kind = r.kind[o]
    C = np.uint64(1 << lg)
    s0 = np.arange(nblocks, dtype=np.uint64) * C
    s1 = s0 + C
    i0 = np.searchsorted(re, s0, side="right")          # first range ending above s0
    i1 = np.searchsorted(rb, s1, side="left") - 1       # last range starting below s1
    cnt = i1 - i0 + 1
    j = np.minimum(i0, len(rb) - 1)
    full = (cnt == 1) & (rb[j] <= s0) & (re[j] >= s1)
    want = np.where(cnt <= 0, 2, 0).astype(np.uint8)
    want[full & (kind[j] == syn.KIND_USER)] = 1
    want[full & (kind[j] == syn.KIND_PROTECTED)] = 3
    want[s1 > np.uint64(2**64 - 1 - lo)] = 0            # ends at (or past) 2^64
    return np.concatenate([want, [2]]).astype(np.uint8)


@pytest.mark.parametrize("log2_page", [12, 21])
def test_cmap_match_blocks(log2_page):
    """The block class map against the per-block classes computed from the ranges, for
    the layouts above plus a table that reaches the top of the address space."""
    lays = list(layouts())
    top = syn.Ranges(np.array([2**64 - 8192, 2**64 - 4096], dtype=np.uint64),
                     np.array([4000, 4095], dtype=np.uint64), np.array([0, 1], np.uint32),
                     np.array([1, 2], np.uint32), {})
    lays.append(("top", top))
    for name, r in lays:
        t, dev = device_table(r, log2_page)
        v = dev.view
        img = dev.buf.cpu().numpy()
        off = v.cmap - dev.address
        words = img[off:off + 4 * ((v.cmap_n + 1 + 15) // 16)].view(np.uint32)
        got = ((words[:, None] >> (2 * np.arange(16, dtype=np.uint32))) & 3).astype(np.uint8).ravel()
        assert v.cmap_log2 >= 8 and v.cmap_n <= 1 << 19, name
        want = block_classes(r, v.lo, v.cmap_log2, v.cmap_n)
        assert (got[:v.cmap_n + 1] == want).all(), name
        assert (want == 1).any() or name == "top", name
