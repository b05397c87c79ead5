"""Guarded streaming kernels (copy / scale / triad) on the GPU vs the oracle."""
import numpy as np
import pytest
import torch

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag
from gpu_util import DEV, assert_log_equal, device_table, new_log

pytestmark = pytest.mark.gpu
OPS = ["copy", "scale", "triad"]
POLICIES = ["poison", "sink", "report"]


def _arena(nbytes):
    buf = torch.empty(nbytes, dtype=torch.uint8, device=DEV)
    assert buf.data_ptr() % 4096 == 0 or buf.data_ptr() % 512 == 0
    return buf


def _view(arena, off, n):
    return arena[off:off + 4 * n].view(torch.float32)


def _fill(n, seed):
    st = syn.Stream(seed, 5)
    b = (st.uniform(n) * 2 - 1).astype(np.float32)
    c = (st.uniform(n) * 2 - 1).astype(np.float32)
    return b, c


@pytest.mark.parametrize("n", [1, 3, 4, 1003, (1 << 20) + 3])
@pytest.mark.parametrize("op", OPS)
def test_stream_no_violation(op, n):
    """With every array inside a user allocation, guarded == unguarded == oracle."""
    r, span, off = syn.stream_layout(n, n_decoys=40, n_prot=8, n_mmio=2, decoy_max=256 * 1024)
    arena = _arena(span)
    base = arena.data_ptr()
    t = r.shifted(base)
    _, dev = device_table(t, 21)
    b, c = _fill(n, n)
    A, B, C = (_view(arena, off[k], n) for k in "abc")
    B.copy_(torch.from_numpy(b))
    C.copy_(torch.from_numpy(c))
    expect = oracle.stream_plain(op, b, c, 3.0)
    for policy in POLICIES:
        A.fill_(-7.0)
        log = new_log()
        ag.agile_stream_launch(op, dev, A, B, C, n, 3.0, policy, log)
        rc, rec = ag.agile_violation_log_read(log)
        assert rc == 0 and rec.count == 0
        got = A.cpu().numpy()
        assert (got.view(np.uint32) == expect.view(np.uint32)).all(), policy
    A.fill_(-7.0)
    ag.agile_stream_launch(op, None, A, B, C, n, 3.0)
    torch.cuda.synchronize()
    assert (A.cpu().numpy().view(np.uint32) == expect.view(np.uint32)).all()


def _hostile_layout(n, base):
    """b overlaps a protected range; c overlaps a hole and an MMIO range; a's user range
    ends before the array does (the tail straddles, then falls into a hole)."""
    nb = 4 * n
    up = lambda x: (x + 255) // 256 * 256
    ob = 0
    oc = up(nb + 8192)
    oa = up(oc + nb + 8192)
    h = nb // 2
    ranges = [
        (ob, 1000, 0, 1), (ob + 1000, 600, 1, 2), (ob + 1600, nb - 1600, 0, 3),
        (oc, h, 0, 4), (oc + h + 64, 48, 2, 5), (oc + h + 4096, nb - h - 4096, 0, 6),
        (oa, int(nb * 0.9) + 6, 0, 7),
    ]
    r = syn._ranges([base + x[0] for x in ranges], [x[1] for x in ranges],
                    [x[2] for x in ranges], [x[3] for x in ranges])
    return r, {"b": base + ob, "c": base + oc, "a": base + oa}, up(oa + nb + 8192)


@pytest.mark.parametrize("n", [4099, (1 << 18) + 1])
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("policy", POLICIES)
def test_stream_violations(op, policy, n):
    _, _, nbytes = _hostile_layout(n, 0)
    arena = _arena(nbytes)
    base = arena.data_ptr()
    r, va, _ = _hostile_layout(n, base)
    _, dev = device_table(r, 12)
    b, c = _fill(n, 77)
    A, B, C = (_view(arena, va[k] - base, n) for k in "abc")
    B.copy_(torch.from_numpy(b))
    C.copy_(torch.from_numpy(c))
    a0 = np.full(n, -5.0, np.float32)
    A.copy_(torch.from_numpy(a0))
    log = new_log(client=3)
    ag.agile_stream_launch(op, dev, A, B, C, n, 3.0, policy, log)
    rc, rec = ag.agile_violation_log_read(log)
    exp, olog = oracle.stream(op, r, va, b, c if op == "triad" else None, a0, 3.0, policy)
    got = A.cpu().numpy()
    assert (got.view(np.uint32) == exp.view(np.uint32)).all()
    assert rc == 1
    assert_log_equal(rec, olog, client=3)


def test_stream_full_size_sampled():
    """The 2^28-element arrays (1 GiB each) in the 1096-range arena: guarded == unguarded
    bit for bit, and sampled elements equal the oracle's arithmetic."""
    n = 1 << 28
    r, span, off = syn.stream_layout(n)
    arena = _arena(span)
    base = arena.data_ptr()
    _, dev = device_table(r.shifted(base), 21)
    A, B, C = (_view(arena, off[k], n) for k in "abc")
    g = torch.Generator(device=DEV).manual_seed(5)
    B.uniform_(-1, 1, generator=g)
    C.uniform_(-1, 1, generator=g)
    ref = torch.empty_like(A)
    idx = torch.from_numpy(syn.Stream(9, 9).below(n, 4096)).to(DEV)
    for op in OPS:
        log = new_log()
        ag.agile_stream_launch(op, dev, A, B, C, n, 3.0, "poison", log)
        ag.agile_stream_launch(op, None, ref, B, C, n, 3.0)
        rc, rec = ag.agile_violation_log_read(log)
        assert rc == 0 and rec.count == 0
        assert torch.equal(A.view(torch.int32), ref.view(torch.int32))
        bs, cs, got = B[idx].cpu().numpy(), C[idx].cpu().numpy(), A[idx].cpu().numpy()
        assert (got == oracle.stream_plain(op, bs, cs, 3.0)).all()


def test_stream_rejects_misaligned_and_bad_args():
    x = torch.zeros(64, dtype=torch.float32, device=DEV)
    with pytest.raises(ag.AgileError) as e:
        ag.agile_stream_launch("copy", None, x.data_ptr() + 4, x, x, 8)
    assert e.value.code == -12
    assert ag.lib().agile_stream_launch(7, None, x.data_ptr(), x.data_ptr(), x.data_ptr(), 8,
                                        1.0, 0, None, None) == -1
    assert ag.lib().agile_stream_launch(0, None, x.data_ptr(), x.data_ptr(), x.data_ptr(), 8,
                                        1.0, 9, None, None) == -1


@pytest.mark.parametrize("chunk", [0, 4, 1 << 12])
@pytest.mark.parametrize("policy", ["poison", "report"])
def test_stream_from_host_equals_one_launch(chunk, policy):
    """The host-array form: chunked copies in, guarded kernels, copies out, on three
    streams. Outputs and the log equal one device launch over the whole arrays, with
    violations in b, c and a, and a ragged tail."""
    n = (1 << 18) + 3
    _, _, nbytes = _hostile_layout(n, 0)
    arena = _arena(nbytes)
    base = arena.data_ptr()
    r, va, _ = _hostile_layout(n, base)
    _, dev = device_table(r, 12)
    b, c = _fill(n, 91)
    A, B, C = (_view(arena, va[k] - base, n) for k in "abc")
    hb = torch.from_numpy(b).pin_memory()
    hc = torch.from_numpy(c).pin_memory()
    for op in OPS:
        a0 = np.full(n, -5.0, np.float32)
        # reference: one device launch
        A.copy_(torch.from_numpy(a0)); B.copy_(hb); C.copy_(hc)
        log = new_log(client=4)
        ag.agile_stream_launch(op, dev, A, B, C, n, 3.0, policy, log)
        rc, rec = ag.agile_violation_log_read(log)
        want = A.cpu().numpy().copy()
        # host form: device inputs cleared first, so they must come from the host
        A.copy_(torch.from_numpy(a0)); B.zero_(); C.zero_()
        ha = torch.empty(n, dtype=torch.float32).pin_memory()
        log2 = new_log(client=4)
        ag.agile_stream_launch_host(op, dev, A, B, C, ha, hb, hc, n, 3.0, policy, log2, chunk)
        rc2, rec2 = ag.agile_violation_log_read(log2)
        assert (ha.numpy().view(np.uint32) == want.view(np.uint32)).all(), op
        assert (rc, rec.count, rec.key, rec.addr, rec.site, rec.verdict, rec.range_id) == \
            (rc2, rec2.count, rec2.key, rec2.addr, rec2.site, rec2.verdict, rec2.range_id), op
        exp, olog = oracle.stream(op, r, va, b, c if op == "triad" else None, a0, 3.0, policy)
        assert (want.view(np.uint32) == exp.view(np.uint32)).all() and rec.count == olog.count


def test_stream_from_host_rejects_bad_chunk():
    x = torch.zeros(64, dtype=torch.float32, device=DEV)
    with pytest.raises(ag.AgileError) as e:
        ag.agile_stream_launch_host("copy", None, x, x, None, None, None, None, 64, chunk_elems=6)
    assert e.value.code == -1
