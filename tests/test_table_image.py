"""The table image on the host (agile_guard_table_image, no GPU): its block class map,
all-user bitmap and open-block descriptors against the same per-block computations the
GPU tests apply to the uploaded image -- the classes and bits from the sorted ranges,
each descriptor's three verdicts from the oracle -- for layouts that include abutting
ranges, MMIO ranges inside one block, a window at the top of the address space and one
over 4 GiB (which has no descriptors)."""
import ctypes

import numpy as np
import pytest

import agile_synth as syn
import paper_2606_06697_b300 as ag
from test_gpu_batch_desc import EMPTY, dense_table, expected_descs, slot_of, top_table
from test_gpu_table import block_classes, brute_bits

LAYOUTS = {
    "batch": syn.batch_table,
    "dense": lambda: dense_table(800, 5),
    "dense_many": lambda: dense_table(6000, 6),
    "top": top_table,
    "table1": syn.table1_apertures,
}


def image(r, lg_page):
    t = ag.agile_guard_table_build(r.base, r.size, r.kind, r.ident, lg_page)
    v, addr, img = t.image()
    return t, v, addr, img


def section(img, addr, ptr, nbytes):
    off = ptr - addr
    assert 0 <= off and off + nbytes <= len(img)
    return img[off:off + nbytes]


@pytest.mark.parametrize("name", sorted(LAYOUTS))
@pytest.mark.parametrize("lg_page", [12, 21])
def test_image_class_map_and_bitmap(name, lg_page):
    r = LAYOUTS[name]()
    t, v, addr, img = image(r, lg_page)
    assert v.bytes == len(img) and v.page - addr == 384
    words = section(img, addr, v.cmap, 4 * ((v.cmap_n + 1 + 15) // 16)).view(np.uint32)
    got = ((words[:, None] >> (2 * np.arange(16, dtype=np.uint32))) & 3).astype(np.uint8).ravel()
    assert (got[:v.cmap_n + 1] == block_classes(r, v.lo, v.cmap_log2, v.cmap_n)).all()
    bw = section(img, addr, v.ubits, 4 * ((v.ubits_n + 1 + 31) // 32)).view(np.uint32)
    bits = ((bw[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(bool).ravel()
    assert (bits[:v.ubits_n + 1] == brute_bits(r, v.lo, v.ubits_log2, v.ubits_n)).all()


@pytest.mark.parametrize("name", sorted(LAYOUTS))
def test_image_descriptors(name):
    r = LAYOUTS[name]()
    t, v, addr, img = image(r, 21)
    window = v.npages << v.log2_page
    if window >= 1 << 32:                          # 32-bit offsets only: no descriptors
        assert not v.cdesc and not v.crange
        return
    assert v.cdesc and 6 <= v.cdesc_log2 <= 12
    want = expected_descs(r, v.lo, v.cmap_log2, v.cmap_n)
    slots = section(img, addr, v.cdesc, 8 << v.cdesc_log2).view(np.uint32).reshape(-1, 2)
    held = {}
    for j, (k, pay) in enumerate(slots.tolist()):
        if k == EMPTY:
            continue
        assert k not in held and k in want
        assert j in (slot_of(k, v.cdesc_k1, v.cdesc_log2), slot_of(k, v.cdesc_k2, v.cdesc_log2))
        assert pay == want[k]
        held[k] = pay
    if 4 * len(want) <= 1 << v.cdesc_log2:
        assert len(held) == len(want)
    else:
        assert len(held) > (1 << v.cdesc_log2) // 4


def test_image_arguments():
    r = syn.batch_table()
    t = ag.agile_guard_table_build(r.base, r.size, r.kind, r.ident, 21)
    v = ag.abi._DevTable()
    buf = np.zeros(t.device_bytes() + 512, dtype=np.uint8)
    off = (-buf.ctypes.data) % 256
    lib = ag.lib()
    p = ctypes.c_void_p(buf.ctypes.data + off)
    assert lib.agile_guard_table_image(t.handle, p, t.device_bytes() - 1, ctypes.byref(v)) == -11
    assert lib.agile_guard_table_image(t.handle, ctypes.c_void_p(buf.ctypes.data + off + 8),
                                       t.device_bytes(), ctypes.byref(v)) == -12
    assert lib.agile_guard_table_image(None, p, t.device_bytes(), ctypes.byref(v)) == -1
    assert lib.agile_guard_table_image(t.handle, p, t.device_bytes(), ctypes.byref(v)) == 0


def test_image_descriptors_all_open_window():
    """A 1 GiB MMIO range with allocations after it: every block of the MMIO range is open
    and describable, far more than the 4096 slots. The build stays quick, fills the slots
    and stores only correct descriptors."""
    import time
    base = 0x7D0000000000
    r = syn._ranges([base, base + (1 << 30), base + (1 << 30) + 8192], [1 << 30, 4096, 100000],
                    [syn.KIND_MMIO, syn.KIND_USER, syn.KIND_PROTECTED], [1, 2, 3])
    t0 = time.perf_counter()
    t, v, addr, img = image(r, 21)
    assert time.perf_counter() - t0 < 10.0
    want = expected_descs(r, v.lo, v.cmap_log2, v.cmap_n)
    assert len(want) > 4 * 4096 and v.cdesc_log2 == 12
    slots = section(img, addr, v.cdesc, 8 << v.cdesc_log2).view(np.uint32).reshape(-1, 2)
    held = [(k, p) for k, p in slots.tolist() if k != EMPTY]
    assert len(held) > 3 * 4096 // 4
    assert all(want[k] == p for k, p in held)
