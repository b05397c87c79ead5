"""PTX-injected guard on the GPU: hand-written PTX, instrumented by the guard pass,
JIT-loaded and run against the oracle (outputs and logs, bit for bit)."""
import ctypes
import os

import numpy as np
import pytest
import torch

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag
from gpu_util import DEV, device_table, new_log
from test_gpu_stream import _fill, _hostile_layout

pytestmark = pytest.mark.gpu
STREAM = open(os.path.join(os.path.dirname(ag.library_path), "ptx", "stream.ptx")).read()
# site numbering of the hand-written kernels -> the oracle's (vector and tail share sites)
SITE_MAP = {"copy": [0, 0, 1, 1, 0, 1, 0, 1], "scale": [0, 0, 1, 1, 0, 1, 0, 1],
            "triad": [0, 0, 1, 1, 2, 2, 0, 1, 2, 0, 1, 2]}


def launch(mod, op, A, B, C, n, s=3.0, grid=148 * 4, block=256):
    args = [ctypes.c_uint64(A.data_ptr()), ctypes.c_uint64(B.data_ptr()),
            ctypes.c_uint64(C.data_ptr()), ctypes.c_uint64(n), ctypes.c_float(s)]
    ag.agile_module_launch(mod, f"agile_ptx_{op}", grid, block, args)


@pytest.fixture(scope="module")
def modules():
    mods = {p: ag.agile_module_load(ag.agile_guard_instrument_ptx(STREAM, p)[0])
            for p in ("poison", "sink", "report")}
    mods["plain"] = ag.agile_module_load(STREAM)
    yield mods
    for m in mods.values():
        m.unload()


@pytest.mark.parametrize("n", [5, 1 << 20])
def test_ptx_no_violation(modules, n):
    r, span, off = syn.stream_layout(n, n_decoys=40, n_prot=8, n_mmio=2, decoy_max=256 * 1024)
    arena = torch.empty(span, dtype=torch.uint8, device=DEV)
    _, dev = device_table(r.shifted(arena.data_ptr()), 21)
    A, B, C = (arena[off[k]:off[k] + 4 * n].view(torch.float32) for k in "abc")
    b, c = _fill(n, 3)
    B.copy_(torch.from_numpy(b))
    C.copy_(torch.from_numpy(c))
    for op in ("copy", "scale", "triad"):
        expect = oracle.stream_plain(op, b, c, 3.0)
        for p in ("poison", "sink", "report", "plain"):
            A.fill_(-1.0)
            log = new_log()
            if p != "plain":
                ag.agile_module_bind(modules[p], dev, log)
            launch(modules[p], op, A, B, C, n)
            rc, rec = ag.agile_violation_log_read(log)
            assert rc == 0 and rec.count == 0, (op, p)
            assert (A.cpu().numpy().view(np.uint32) == expect.view(np.uint32)).all(), (op, p)


@pytest.mark.parametrize("n", [4099, (1 << 18) + 1])
@pytest.mark.parametrize("policy", ["poison", "sink", "report"])
def test_ptx_violations(modules, policy, n):
    _, _, nbytes = _hostile_layout(n, 0)
    arena = torch.empty(nbytes, dtype=torch.uint8, device=DEV)
    base = arena.data_ptr()
    r, va, _ = _hostile_layout(n, base)
    _, dev = device_table(r, 12)
    b, c = _fill(n, 77)
    A, B, C = (arena[va[k] - base:va[k] - base + 4 * n].view(torch.float32) for k in "abc")
    B.copy_(torch.from_numpy(b))
    C.copy_(torch.from_numpy(c))
    for op in ("copy", "scale", "triad"):
        a0 = np.full(n, -5.0, np.float32)
        A.copy_(torch.from_numpy(a0))
        log = new_log(client=9)
        ag.agile_module_bind(modules[policy], dev, log)
        launch(modules[policy], op, A, B, C, n)
        rc, rec = ag.agile_violation_log_read(log)
        exp, olog = oracle.stream(op, r, va, b, c if op == "triad" else None, a0, 3.0, policy)
        assert (A.cpu().numpy().view(np.uint32) == exp.view(np.uint32)).all(), op
        assert rc == 1 and rec.count == olog.count and rec.client == 9
        assert (rec.key, rec.addr, rec.width, rec.verdict, rec.range_id) == \
            (olog.key, olog.addr, olog.width, olog.verdict, olog.range_id), (op, rec, olog)
        assert SITE_MAP[op][rec.site] == olog.site


def test_ptx_class_map_tier(modules):
    """Arrays whose edges sit 256 bytes into 4 KiB bitmap blocks, each between two 256-byte
    protected ranges: the bitmap's edge blocks are not all user, the class map's 256-byte
    blocks are, so those accesses are allowed by the second inline test. Outputs equal the
    plain module's and nothing is logged; one element past b's end is then denied."""
    n = 3 * 1024 + 64                                  # 12,544 bytes per array
    nb = 4 * n
    ob, oc, oa = 4096 + 256, 5 * 4096 + 256, 9 * 4096 + 256
    ranges = []
    for k, o in enumerate((ob, oc, oa)):
        ranges += [(o - 256, 256, 1, 10 + k), (o, nb, 0, 20 + k), (o + nb, 256, 1, 30 + k)]
    arena = torch.zeros(13 * 4096, dtype=torch.uint8, device=DEV)
    base = arena.data_ptr()
    r = syn._ranges([base + x[0] for x in ranges], [x[1] for x in ranges],
                    [x[2] for x in ranges], [x[3] for x in ranges])
    t, dev = device_table(r, 12)
    assert t.geometry()[0] == 12
    A, B, C = (arena[o:o + nb].view(torch.float32) for o in (oa, ob, oc))
    b, c = _fill(n, 5)
    B.copy_(torch.from_numpy(b))
    C.copy_(torch.from_numpy(c))
    for op in ("copy", "scale", "triad"):
        expect = oracle.stream_plain(op, b, c, 3.0)
        A.fill_(-1.0)
        log = new_log()
        ag.agile_module_bind(modules["poison"], dev, log)
        launch(modules["poison"], op, A, B, C, n)
        rc, rec = ag.agile_violation_log_read(log)
        assert rc == 0 and rec.count == 0, op
        assert (A.cpu().numpy().view(np.uint32) == expect.view(np.uint32)).all(), op
    # one more element: b's and c's last reads and a's last write land in the protected tails
    A.fill_(-1.0)
    log = new_log()
    ag.agile_module_bind(modules["poison"], dev, log)
    launch(modules["poison"], "copy", arena[oa:oa + nb + 4].view(torch.float32),
           arena[ob:ob + nb + 4].view(torch.float32), C, n + 1)
    rc, rec = ag.agile_violation_log_read(log)
    assert rc == 1 and rec.count == 2 and rec.verdict == 1
    assert rec.addr == base + ob + nb and rec.range_id == 30


EXITS = """
.version 9.0
.target sm_103a
.address_size 64
.visible .entry agile_ptx_exits(.param .u64 p_a, .param .u64 p_n)
{
    .reg .pred %p<4>;
    .reg .b32 %r<6>;
    .reg .b64 %rd<6>;
    ld.param.u64 %rd1, [p_a];
    ld.param.u64 %rd2, [p_n];
    mov.u32 %r1, %tid.x;
    mov.u32 %r2, %ctaid.x;
    mov.u32 %r3, %ntid.x;
    mad.lo.u32 %r4, %r2, %r3, %r1;
    cvt.u64.u32 %rd3, %r4;
    setp.ge.u64 %p1, %rd3, %rd2;
    @%p1 bra $DONE;
    shl.b64 %rd4, %rd3, 2;
    add.s64 %rd5, %rd1, %rd4;
    st.global.u32 [%rd5], %r4;
    and.b32 %r5, %r4, 3;
    setp.eq.u32 %p2, %r5, 1;
    @%p2 ret;
    setp.eq.u32 %p3, %r5, 2;
    @%p3 exit;
    st.global.u32 [%rd5+4], %r4;
$DONE:
    ret;
}
"""


@pytest.mark.parametrize("policy", ["poison", "report"])
def test_ptx_violations_merged_at_every_exit(policy):
    """Thread i stores a[i]; threads with i mod 4 = 1 then return and those with
    i mod 4 = 2 exit; the rest also store a[i + 1]. The array runs past its user range
    into a protected one, so denials land before each way out. The log -- merged from
    registers before each ret and exit -- holds the oracle's count and, for the smallest
    denied address, its record (site 0: the first store)."""
    n, m = 5000, 3333                                   # threads; elements inside the range
    arena = torch.zeros(8 << 20, dtype=torch.uint8, device=DEV)
    base = arena.data_ptr()
    a = base + 4096
    r = syn._ranges([a, a + 4 * m], [4 * m, 2 << 20], [0, 1], [7, 8])
    t, dev = device_table(r, 12)
    mod = ag.agile_module_load(ag.agile_guard_instrument_ptx(EXITS, policy)[0])
    try:
        log = new_log(client=3)
        ag.agile_module_bind(mod, dev, log)
        ag.agile_module_launch(mod, "agile_ptx_exits", (n + 255) // 256, 256,
                               [ctypes.c_uint64(a), ctypes.c_uint64(n)])
        rc, rec = ag.agile_violation_log_read(log)
    finally:
        mod.unload()
    i = np.arange(n, dtype=np.uint64)
    second = i[(i % 4 != 1) & (i % 4 != 2)]
    addrs = np.concatenate([a + 4 * i, a + 4 * (second + 1)]).astype(np.uint64)
    sites = np.concatenate([np.zeros(n, np.uint32), np.ones(len(second), np.uint32)])
    v, rid, olog = oracle.check_batch(r, addrs, np.full(len(addrs), 4, np.uint8), method="sorted")
    denied = v != 0
    k = np.lexsort((sites[denied], addrs[denied]))[0]   # smallest address, then site
    assert rc == 1 and rec.count == int(denied.sum()) == olog.count and rec.client == 3
    assert (rec.addr, rec.site, rec.verdict, rec.range_id, rec.width) == \
        (int(addrs[denied][k]), int(sites[denied][k]), int(v[denied][k]), int(rid[denied][k]), 4)
    # every allowed store landed: a[j] holds j, or j - 1 where thread j - 1 stored it second
    got = arena[4096:4096 + 4 * m].view(torch.int32).cpu().numpy().astype(np.int64)
    j = np.arange(m)
    assert ((got == j) | ((got == j - 1) & np.isin((j - 1) % 4, (0, 3)))).all()


def test_ptx_launch_refused_until_bound():
    m = ag.agile_module_load(ag.agile_guard_instrument_ptx(STREAM, "poison")[0])
    x = torch.zeros(64, dtype=torch.float32, device=DEV)
    with pytest.raises(ag.AgileError) as e:
        launch(m, "copy", x, x, x, 64, grid=1, block=32)
    assert e.value.code == -1
    with pytest.raises(ag.AgileError):
        ag.agile_module_launch(m, "no_such_kernel", 1, 32, [])
    m.unload()


IRREGULAR = open(os.path.join(os.path.dirname(ag.library_path), "ptx", "irregular.ptx")).read()
IRR_SITES = {"gather": [0, 1, 2, 2, 2, 2, 3, 0, 2, 3], "scatter": [0, 1, 2, 2, 2, 2, 0, 2],
             "hist": [0, 1, 2, 2, 2, 2, 0, 2]}


@pytest.mark.parametrize("policy", ["poison", "sink", "report"])
@pytest.mark.parametrize("n", [7, 40_003])
def test_ptx_irregular_parity(policy, n):
    from test_gpu_irregular import put, setup
    mod = ag.agile_module_load(ag.agile_guard_instrument_ptx(IRREGULAR, policy)[0])
    try:
        for kind in ("gather", "scatter", "hist"):
            r, span, off, idx, key, bad, host, arena, base = setup(n, frac_bad=0.05)
            put(host, off["idx"], key if kind == "hist" else idx)
            t = r.shifted(base)
            _, dev = device_table(t, 16)
            arena.copy_(torch.from_numpy(host))
            log = new_log(client=5)
            ag.agile_module_bind(mod, dev, log)
            target = off["bins"] if kind == "hist" else off["t"]
            args = [ctypes.c_uint64(base + off["idx"]), ctypes.c_uint64(base + target),
                    ctypes.c_uint64(base + off["out"]), ctypes.c_uint64(n)]
            ag.agile_module_launch(mod, f"agile_ptx_{kind}", 148 * 2, 256, args)
            rc, rec = ag.agile_violation_log_read(log)
            va = {"t": base + target, "idx": base + off["idx"], "out": base + off["out"]}
            olog = oracle.irregular(kind, t, host, base, va, n, policy)
            assert (arena.cpu().numpy() == host).all(), kind
            assert rec.count == olog.count and rec.client == 5
            if olog.count:
                assert (rec.key, rec.addr, rec.width, rec.verdict, rec.range_id) == \
                    (olog.key, olog.addr, olog.width, olog.verdict, olog.range_id), kind
                assert IRR_SITES[kind][rec.site] == olog.site
    finally:
        mod.unload()


@pytest.mark.parametrize("n", [7, 40_003])
def test_ptx_irregular_remap_parity(n):
    """The pass's REMAP_OR policy on the irregular PTX kernels vs the oracle."""
    from test_gpu_irregular import assert_remap_arena, put, remap_setup, remap_table
    half = 1 << 20
    mod = ag.agile_module_load(ag.agile_guard_instrument_ptx(IRREGULAR, "remap")[0])
    try:
        for kind in ("gather", "scatter", "hist"):
            r, off, idx, key, cls, host, arena, base = remap_setup(n, half)
            put(host, off["idx"], key if kind == "hist" else idx)
            _, dev = remap_table(r, base, half, 16)
            arena.copy_(torch.from_numpy(host))
            log = new_log(client=6)
            ag.agile_module_bind(mod, dev, log)
            target = off["bins"] if kind == "hist" else off["t"]
            args = [ctypes.c_uint64(base + off["idx"]), ctypes.c_uint64(base + target),
                    ctypes.c_uint64(base + off["out"]), ctypes.c_uint64(n)]
            ag.agile_module_launch(mod, f"agile_ptx_{kind}", 148 * 2, 256, args)
            rc, rec = ag.agile_violation_log_read(log)
            va = {"t": base + target, "idx": base + off["idx"], "out": base + off["out"]}
            olog = oracle.irregular(kind, r.shifted(base), host, base, va, n, "remap", remap=half)
            assert_remap_arena(kind, arena.cpu().numpy(), host, off, idx, cls, half)
            assert rec.count == olog.count and rec.client == 6
            if olog.count:
                assert (rec.key, rec.addr, rec.width, rec.verdict, rec.range_id) == \
                    (olog.key, olog.addr, olog.width, olog.verdict, olog.range_id), kind
                assert IRR_SITES[kind][rec.site] == olog.site
    finally:
        mod.unload()


# ---------------------------------------------------------------- aperture rule


def _aps(r):
    return (r.base, r.size, r.kind, r.ident)


@pytest.mark.parametrize("policy", ["poison", "sink", "report"])
def test_ptx_aperture_stream(policy):
    """The pass with apertures (no table bound): a protected and an MMIO window over b and
    c and a protected window over a; the straddling tail of a and the hole in c, which the
    table rule denies, pass."""
    n = 4099
    _, _, nbytes = _hostile_layout(n, 0)
    arena = torch.empty(nbytes, dtype=torch.uint8, device=DEV)
    base = arena.data_ptr()
    r, va, _ = _hostile_layout(n, base)
    keep = r.kind != syn.KIND_USER
    ap = syn._ranges(list(r.base[keep]) + [va["a"] + 4096], list(r.size[keep]) + [256],
                     list(r.kind[keep]) + [syn.KIND_PROTECTED], list(r.ident[keep]) + [8])
    mod = ag.agile_module_load(ag.agile_guard_instrument_ptx(STREAM, policy, apertures=_aps(ap))[0])
    try:
        b, c = _fill(n, 78)
        A, B, C = (arena[va[k] - base:va[k] - base + 4 * n].view(torch.float32) for k in "abc")
        B.copy_(torch.from_numpy(b))
        C.copy_(torch.from_numpy(c))
        for op in ("copy", "scale", "triad"):
            a0 = np.full(n, -5.0, np.float32)
            A.copy_(torch.from_numpy(a0))
            log = new_log(client=11)
            ag.agile_module_bind(mod, None, log)
            launch(mod, op, A, B, C, n)
            rc, rec = ag.agile_violation_log_read(log)
            exp, olog = oracle.stream(op, ap, va, b, c if op == "triad" else None, a0, 3.0, policy,
                                      rule="aperture")
            assert (A.cpu().numpy().view(np.uint32) == exp.view(np.uint32)).all(), op
            assert rc == 1 and rec.count == olog.count and rec.client == 11
            assert (rec.key, rec.addr, rec.width, rec.verdict, rec.range_id) == \
                (olog.key, olog.addr, olog.width, olog.verdict, olog.range_id), (op, rec, olog)
            assert SITE_MAP[op][rec.site] == olog.site
    finally:
        mod.unload()


@pytest.mark.parametrize("policy", ["poison", "sink", "report"])
@pytest.mark.parametrize("n", [7, 40_003])
def test_ptx_aperture_irregular(policy, n):
    """Irregular kernels under the aperture rule on the shadow/user layout, with extra
    accesses into a hole (allowed by the aperture rule)."""
    from test_gpu_irregular import put, remap_setup
    half = 1 << 20
    for kind in ("gather", "scatter", "hist"):
        r, off, idx, key, cls, host, arena, base = remap_setup(n, half)
        t = r.shifted(base)
        keep = t.kind != syn.KIND_USER
        ap = syn._ranges(t.base[keep], t.size[keep], t.kind[keep], t.ident[keep])
        # the apertures are compiled into the module, so each arena gets its own
        mod = ag.agile_module_load(ag.agile_guard_instrument_ptx(IRREGULAR, policy, apertures=_aps(ap))[0])
        try:
            ne = half // 4
            hole = np.arange(0, n, 13)
            idx, key = idx.copy(), key.copy()
            idx[hole] = 2 * ne + hole % 4096            # the hole at [3 half, 4 half)
            key[hole] = -2 * ne + hole % 4096
            put(host, off["idx"], key if kind == "hist" else idx)
            arena.copy_(torch.from_numpy(host))
            log = new_log(client=12)
            ag.agile_module_bind(mod, None, log)
            target = off["bins"] if kind == "hist" else off["t"]
            args = [ctypes.c_uint64(base + off["idx"]), ctypes.c_uint64(base + target),
                    ctypes.c_uint64(base + off["out"]), ctypes.c_uint64(n)]
            ag.agile_module_launch(mod, f"agile_ptx_{kind}", 148 * 2, 256, args)
            rc, rec = ag.agile_violation_log_read(log)
            va = {"t": base + target, "idx": base + off["idx"], "out": base + off["out"]}
            olog = oracle.irregular(kind, ap, host, base, va, n, policy, rule="aperture")
            assert (arena.cpu().numpy() == host).all(), kind
            assert rec.count == olog.count and rec.client == 12
            if olog.count:
                assert (rec.key, rec.addr, rec.width, rec.verdict, rec.range_id) == \
                    (olog.key, olog.addr, olog.width, olog.verdict, olog.range_id), kind
                assert IRR_SITES[kind][rec.site] == olog.site
        finally:
            mod.unload()


def test_ptx_bind_without_table_only_for_aperture_modules():
    m = ag.agile_module_load(ag.agile_guard_instrument_ptx(STREAM, "poison")[0])
    with pytest.raises(ag.AgileError):
        ag.agile_module_bind(m, None, new_log())
    m.unload()
