"""Host-side checks that need no GPU: the library loads and exports every entry point
the header declares; table rules and API-time validation match the oracle."""
import os
import re
import subprocess

import numpy as np
import pytest

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared():
    names = []
    for h in HEADERS:
        names += re.findall(r"^AGILE_API\s+[\w\s\*]+?\b(agile_\w+)\s*\(", open(h).read(), re.M)
    return names


def test_library_exports_every_declared_symbol():
    names = declared()
    assert len(names) >= 18
    L = ag.lib()
    for name in names:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", ag.library_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (agile_\w+)", out))
    assert set(names) == exported


def test_violation_list_arguments():
    """The bounded list's size formula and its argument checks, which run before any CUDA
    call."""
    import ctypes
    assert ag.list_bytes(0) == 16 and ag.list_bytes(3) == 16 + 3 * 32
    L = ag.lib()
    assert L.agile_violation_list_attach(None, None, 4, None) == -1          # no log
    assert L.agile_violation_list_attach(0x1000, 0x2000, 0, None) == -1      # capacity 0
    assert L.agile_violation_list_attach(0x1008, 0x2000, 4, None) == -12     # log alignment
    assert L.agile_violation_list_attach(0x1000, 0x2008, 4, None) == -12     # list alignment
    n_out, n_seen = ctypes.c_size_t(), ctypes.c_uint64()
    assert L.agile_violation_list_read(None, 0x2000, None, 0, ctypes.byref(n_out),
                                       ctypes.byref(n_seen), None) == -1
    assert L.agile_violation_list_read(0x1000, 0x2000, None, 4, ctypes.byref(n_out),
                                       ctypes.byref(n_seen), None) == -1      # no room given


def test_strerror_and_version():
    assert ag.agile_version() == 0x000100
    assert "overlap" in ag.agile_strerror(-2)
    assert ag.agile_strerror(12345) == "unknown error"


ERR = {1: -3, 2: -4, 3: -2, 4: -5}


@pytest.mark.parametrize("case", [
    ([0, 16, 32], [16, 16, 1], [0, 0, 1]),
    ([0, 15], [16, 4], [0, 1]),
    ([0], [0], [0]),
    ([2**64 - 1], [1], [0]),
    ([2**64 - 2], [1], [0]),
    ([0], [1], [3]),
    ([100, 0, 50], [10, 50, 50], [2, 1, 0]),
    ([100, 0, 50], [10, 51, 50], [2, 1, 0]),
])
def test_table_rules_match_oracle(case):
    base, size, kind = case
    r = syn._ranges(base, size, kind, list(range(len(base))))
    want = oracle.table_check(r)
    if want == 0:
        ag.agile_guard_table_build(r.base, r.size, r.kind, r.ident)
    else:
        with pytest.raises(ag.AgileError) as e:
            ag.agile_guard_table_build(r.base, r.size, r.kind, r.ident)
        assert e.value.code == ERR[want]


def test_table_page_geometry():
    r = syn.batch_table()
    t = ag.agile_guard_table_build(r.base, r.size, r.kind, r.ident, 21)
    lg, npages = t.geometry()
    first, last = int(r.base.min()) >> 21, (int((r.base + r.size).max()) - 1) >> 21
    assert lg == 21 and npages == last - first + 1 <= 512   # pages from first to last range
    t1 = syn.table1_apertures()
    big = ag.agile_guard_table_build(t1.base, t1.size, t1.kind, t1.ident, 12)
    lg, npages = big.geometry()
    assert npages <= 1 << 26 and lg > 12       # page size raised to bound the map
    with pytest.raises(ag.AgileError):
        ag.agile_guard_table_build(t1.base, t1.size, t1.kind, t1.ident, 11)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_validate_args_matches_oracle(seed):
    """API-time validation (arbitrary byte counts) against the oracle's linear scan."""
    t = syn.batch_table(seed=syn.SEED_BASE + 40 + seed)
    st = syn.Stream(seed, 40)
    base, size = t.base.astype(np.int64), t.size.astype(np.int64)
    n = 20000
    j = st.below(len(t), n)
    off = st.below(size[j] + 64, n) - 32
    ptr = (base[j] + off).astype(np.uint64)
    nbytes = np.where(st.below(4, n) == 0, 0, st.log_uniform(1, 1 << 24, n)).astype(np.uint64)
    tbl = ag.agile_guard_table_build(t.base, t.size, t.kind, t.ident, 21)
    rc, v, rid = ag.agile_validate_args(tbl, ptr, nbytes)
    ov, orid = oracle.validate(t, ptr, nbytes)
    assert (v == ov).all() and (rid == orid).all()
    assert rc == (1 if (ov != 0).any() else 0)
    # the exact whole allocation passes
    rc, v, _ = ag.agile_validate_args(tbl, t.base, t.size)
    assert ((v == 0) == (t.kind == 0)).all()


def test_validate_args_table1_golden():
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "table1_apertures.txt")):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            if f[0] == "v":
                rows.append((int(f[1], 16), int(f[2], 0), oracle.VERDICT_NAMES.index(f[3])))
    t = syn.table1_apertures()
    tbl = ag.agile_guard_table_build(t.base, t.size, t.kind, t.ident)
    _, v, _ = ag.agile_validate_args(tbl, [r[0] for r in rows], [r[1] for r in rows])
    assert v.tolist() == [r[2] for r in rows]


def test_upload_without_gpu_reports_cuda_error():
    """Host-only machine: the library loads; a device call fails with AGILE_ERR_CUDA, not a crash."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    t = ag.agile_guard_table_build([0], [16], [0], [1])
    with pytest.raises(ag.AgileError) as e:
        t.upload(0x100000)
    assert e.value.code in (-7,)


def test_python_struct_mirrors_match_the_header():
    """ctypes mirrors of the public structs have the sizes the C header gives them."""
    import ctypes
    from paper_2606_06697_b300 import abi
    src = r"""
#include <stdio.h>
#include "agile_guard.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu ", sizeof(agile_range_t), sizeof(agile_dev_table_t),
         sizeof(agile_violation_record_t), sizeof(agile_work_t), sizeof(agile_batch_config_t),
         sizeof(agile_request_t), sizeof(agile_completion_t), sizeof(agile_worker_config_t));
  return 0;
}
"""
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    mirrors = [abi._Range, abi._DevTable, abi._Record, abi.Work, abi.BatchConfig, abi.Request,
               abi.Completion, abi.WorkerConfig]
    assert sizes == [ctypes.sizeof(m) for m in mirrors]


@pytest.mark.parametrize("seed", [3, 4])
def test_validate_dma_matches_oracle(seed):
    t = syn.batch_table(seed=syn.SEED_BASE + 80 + seed)
    st = syn.Stream(seed, 81)
    n = 5000
    j = st.below(len(t), n)
    base, size = t.base.astype(np.int64), t.size.astype(np.int64)
    mode = st.below(4, n)
    ptr = np.where(mode == 3, base[j] + st.below(size[j], n), base[j])
    nb = np.where(mode == 0, size[j], np.where(mode == 1, size[j] - 1, st.log_uniform(1, 1 << 20, n)))
    tbl = ag.agile_guard_table_build(t.base, t.size, t.kind, t.ident, 21)
    rc, v, rid = ag.agile_validate_dma(tbl, ptr.astype(np.uint64), np.maximum(nb, 0).astype(np.uint64))
    ov, orid = oracle.validate_exact(t, ptr.astype(np.uint64), np.maximum(nb, 0).astype(np.uint64))
    assert (v == ov).all() and (rid == orid).all()
    assert (v == 0).any() and (v == 6).any()


@pytest.mark.parametrize("bad,code", [
    (syn._ranges([0xF0000000000] * 5, [16] * 5, [2] * 5, [1] * 5), -11),        # over the maximum
    (syn._ranges([0x1000], [16], [syn.KIND_USER], [1]), -5),                     # a user aperture
    (syn._ranges([0x1000, 0x1008], [16, 16], [syn.KIND_MMIO] * 2, [1, 2]), -2),  # overlap
    (syn._ranges([0x1000], [0], [syn.KIND_MMIO], [1]), -3),                      # empty
    (syn._ranges([2**64 - 8], [16], [syn.KIND_MMIO], [1]), -4),                  # end past 2^64 - 1
])
def test_aperture_set_rejected_before_launch(bad, code):
    """The aperture set is validated on the host before anything reaches the device."""
    with pytest.raises(ag.AgileError) as e:
        ag.agile_aperture_check_batch((bad.base, bad.size, bad.kind, bad.ident), 0x1000, 0x2000, 8,
                                      0x3000)
    assert e.value.code == code


def test_host_array_and_selftest_arguments_checked_before_launch():
    """Argument errors of the host-array entry point and the bounded-wait self-test come
    back from the host side, before anything is queued on a device."""
    lib = ag.lib()
    assert lib.agile_stream_launch_host(7, None, 0x1000, 0x1000, None, None, None, None, 64,
                                        1.0, 0, None, 0, None) == -1          # unknown op
    assert lib.agile_stream_launch_host(0, None, 0x1000, 0x1000, None, None, None, None, 64,
                                        1.0, 0, None, 6, None) == -1          # chunk % 4 != 0
    assert lib.agile_stream_launch_host(0, None, 0x1000, 0x1000, None, None, None, None, 0,
                                        1.0, 0, None, 0, None) == 0           # nothing to do
    assert lib.agile_stream_launch_host(2, None, 0x1000, 0x1000, None, None, None, None, 64,
                                        1.0, 0, None, 0, None) == -1          # triad without c
    # Every chunk's checks are made once, up front: a misaligned array or log, or a bad
    # policy, is refused before any stream, event or copy exists (on this host, with no
    # device, any CUDA call would come back as AGILE_ERR_CUDA instead).
    assert lib.agile_stream_launch_host(2, None, 0x1000, 0x1000, 0x2008, None, None, None, 1 << 20,
                                        1.0, 0, None, 1 << 16, None) == -12   # c misaligned
    assert lib.agile_stream_launch_host(0, None, 0x1004, 0x1000, None, None, None, None, 64,
                                        1.0, 0, None, 0, None) == -12         # a misaligned
    assert lib.agile_stream_launch_host(0, None, 0x1000, 0x1000, None, None, None, None, 64,
                                        1.0, 0, 0x3008, 0, None) == -12       # log misaligned
    assert lib.agile_stream_launch_host(0, None, 0x1000, 0x1000, None, None, None, None, 64,
                                        1.0, 9, None, 0, None) == -1          # unknown policy
    assert lib.agile_selftest_bounded_waits(0x1000, 0x2000, 0, 0x3000, None) == -1
    assert lib.agile_selftest_bounded_waits(0x1000, 0x2000, 2_000_000, 0x3000, None) == -1
    assert lib.agile_selftest_bounded_waits(0x1008, 0x2000, 100, 0x3000, None) == -12


def test_auto_page_size():
    """AGILE_PAGE_AUTO: the largest page at which 95% of the user bytes lie in pages wholly
    inside one user range. The stress stripes (60 KiB user + 4 KiB protected) need 4 KiB
    pages; the 4 MiB + 64 KiB stripes are 95% pure at 256 KiB; Table I's huge apertures at
    2 MiB; every choice keeps the page map within 2^24 entries."""
    cases = [(syn.irregular_layout(1 << 20, 1 << 18, 60 << 10, 4 << 10, 1 << 10)[0], 12),
             (syn.irregular_layout(1 << 20)[0], 18),
             (syn.table1_apertures(), 21)]
    for r, want in cases:
        rr = r.shifted(0x7E0000000000) if int(r.base.max()) < 2**40 else r
        t = ag.agile_guard_table_build(rr.base, rr.size, rr.kind, rr.ident, 0)
        lg, npages = t.geometry()
        assert lg == want and npages <= 1 << 24
        # and the rule by hand at the choice and one step coarser
        o = np.argsort(rr.base)
        base, end = rr.base[o].astype(object), (rr.base[o] + rr.size[o]).astype(object)
        user = rr.kind[o] == syn.KIND_USER

        def share(g):
            G = 1 << g
            pure = sum(max(0, (int(e) // G) - (-(-int(b) // G))) * G
                       for b, e, u in zip(base, end, user) if u)
            return pure / sum(int(e) - int(b) for b, e, u in zip(base, end, user) if u)
        assert share(lg) >= 0.95 or lg == 12
        if lg < 21:
            assert share(lg + 1) < 0.95
