"""The allocation-free batched launch (agile_batch_launch_static).

Some callers cannot allocate device memory: a worker whose whole budget is already
handed out by its admission accounting, code that must not risk the implicit device
synchronization of cudaMalloc/cudaFree, or a plugin whose host gives it no allocator.
This entry point keeps the batch's scratch in a fixed array inside the library; the
caller still provides every input and output. Its results must equal the regular
batched launch, whose scratch lives in a caller-provided buffer. This file is collected
last and also passes when run on its own in a fresh process (its first call performs the
per-device set-up).
"""
import ctypes

import numpy as np
import pytest
import torch

import agile_synth as syn
import paper_2606_06697_b300 as ag
from paper_2606_06697_b300.clients import ClientSet

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def snapshot(cs):
    out = []
    for o, rec in cs.outputs():
        out.append((o.view(np.uint32).tobytes(),
                    (rec.count, rec.key, rec.addr, rec.width, rec.verdict, rec.site,
                     rec.range_id, rec.client, rec.status)))
    return out


def test_static_launch_equals_buffer_launch_twice():
    specs = syn.client_specs(20, seed=syn.SEED_BASE + 50, median=48 * 1024, lo=4 * 1024,
                             hi=512 * 1024, table_lo=8, table_hi=300)
    cs = ClientSet(specs, DEV, log2_pages=(16,), frac_bad=0.01)
    n = len(cs.clients)
    items = cs.work(0)
    buf = torch.empty(ag.agile_batch_device_bytes(n), dtype=torch.uint8, device=DEV)
    ag.agile_batch_upload(items, 4096, buf)
    ag.agile_batch_launch(buf, n, 4096)
    torch.cuda.synchronize()
    want = snapshot(cs)
    assert any(w[1][0] for w in want)              # some violations were logged
    for _ in range(2):                             # two calls in a row share the array
        cs.reset()
        arr = (ag.Work * n)(*items)
        cfg = ag.abi.BatchConfig(4096, 1, 2, 0)
        rc = ag.lib().agile_batch_launch_static(arr, n, 4096, ctypes.byref(cfg), None)
        assert rc == 0
        torch.cuda.synchronize()
        assert snapshot(cs) == want


def test_static_launch_full_array_on_a_stream():
    """AGILE_BATCH_STATIC_MAX_ITEMS items -- the work list and prefix sums fill the fixed
    array -- on a non-default stream, twice: equal to the buffer launch of the same list.
    The list repeats a few clients' work; histogram items then count several times, the
    same number of times on both paths."""
    specs = syn.client_specs(16, seed=syn.SEED_BASE + 51, median=16 * 1024, lo=4 * 1024,
                             hi=64 * 1024, table_lo=8, table_hi=64)
    cs = ClientSet(specs, DEV, log2_pages=(16,), frac_bad=0.01)
    base = cs.work(0)
    m = ag.BATCH_STATIC_MAX_ITEMS
    items = [base[k % len(base)] for k in range(m)]
    st = torch.cuda.Stream(device=DEV)
    cs.reset()
    buf = torch.empty(ag.agile_batch_device_bytes(m), dtype=torch.uint8, device=DEV)
    torch.cuda.synchronize()                       # the resets (default stream) come first
    ag.agile_batch_upload(items, 4096, buf, st)
    ag.agile_batch_launch(buf, m, 4096, stream=st)
    st.synchronize()
    want = snapshot(cs)
    arr = (ag.Work * m)(*items)
    cfg = ag.abi.BatchConfig(4096, 1, 2, 0)
    for _ in range(2):
        cs.reset()
        torch.cuda.synchronize()
        rc = ag.lib().agile_batch_launch_static(arr, m, 4096, ctypes.byref(cfg),
                                                ctypes.c_void_p(st.cuda_stream))
        assert rc == 0
        st.synchronize()
        assert snapshot(cs) == want


def test_static_launch_rejects_too_many_items():
    items = [ag.Work() for _ in range(ag.BATCH_STATIC_MAX_ITEMS + 1)]
    with pytest.raises(ag.AgileError) as e:
        ag.agile_batch_launch_static(items, 4096)
    assert e.value.code == -11
