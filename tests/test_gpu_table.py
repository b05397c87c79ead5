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
