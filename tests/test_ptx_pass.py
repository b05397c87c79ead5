"""The PTX guard pass on hand-written PTX, checked as text (no GPU): every global
access gets a guard, the policies emit what they should, skipped functions and other
state spaces stay untouched, uncoverable forms are rejected, and the output assembles
for sm_103a (ptxas)."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

import paper_2606_06697_b300 as ag

PTX_DIR = os.path.join(os.path.dirname(ag.library_path), "ptx")
STREAM = open(os.path.join(PTX_DIR, "stream.ptx")).read()
HDR = ".version 9.0\n.target sm_103a\n.address_size 64\n"


MERGE_AT_ONCE = "@!%__agp2 call __agile_guard_merge, (__agmk, __agmi, __agmc);"
KEEP_IN_REGS = "@%__agp2 add.u32 %__agc, %__agc, 1;"


def slow_paths(text):
    """Labels that end each inlined copy of the slow path."""
    return re.findall(r"\$__AGC\d+_END:", text)


def kernel(body, regs=".reg .b64 %rd<8>;\n.reg .f32 %f<8>;\n.reg .b32 %r<8>;\n.reg .pred %p<4>;",
           name="k"):
    return HDR + f".visible .entry {name}(.param .u64 p0)\n{{\n{regs}\nld.param.u64 %rd1, [p0];\n{body}\nret;\n}}\n"


def assemble(ptx):
    if shutil.which("ptxas") is None:
        pytest.skip("ptxas not found")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "m.ptx")
        open(src, "w").write(ptx)
        r = subprocess.run(["ptxas", "-arch=sm_103a", src, "-o", os.path.join(d, "m.cubin")],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def sites(text):
    return re.findall(r"// agile guard: site (\d+), (\S+), (\d+) bytes", text)


@pytest.mark.parametrize("policy", ["poison", "sink", "report", "trap", "remap"])
def test_stream_kernels_every_access_guarded(policy):
    out, rep = ag.agile_guard_instrument_ptx(STREAM, policy)
    n_acc = len(re.findall(r"\b(?:ld|st)\.global\.", STREAM))
    assert rep == {"functions": 3, "guarded": n_acc, "generic_guarded": 0, "skipped": 0}
    s = sites(out)
    assert len(s) == n_acc == 28
    assert [x[1] for x in s[:6]] == ["ld.global.v4.f32", "ld.global.v4.f32", "st.global.v4.f32",
                                     "st.global.v4.f32", "ld.global.v4.f32", "st.global.v4.f32"]
    assert [int(x[2]) for x in s[:8]] == [16, 16, 16, 16, 16, 16, 4, 4]
    slow = 2 * n_acc if policy == "remap" else n_acc      # remap re-checks address | mask
    assert len(slow_paths(out)) == slow                      # the slow path, inlined
    assert "__agile_guard_check" not in out
    # entry functions keep violations in registers and merge them before each ret; under
    # TRAP every violation is merged at once, as a trap ends the kernel
    merged_at_once = policy == "trap"
    assert out.count(MERGE_AT_ONCE) == (n_acc if merged_at_once else 0)
    assert out.count(KEEP_IN_REGS) == (0 if merged_at_once else n_acc)
    rets = len(re.findall(r"\bret;", STREAM))
    flushes = out.count("call __agile_guard_flush, (__agfc, __agfk, __agfi);")
    assert flushes == (0 if merged_at_once else rets + 3)     # each ret, and each body's end
    # the class-map test sits between the bitmap test and the call, once per access
    assert out.count("ld.global.nc.v2.u32 {%__agr0, %__agr1}, [%__agT7+136];") == n_acc
    assert out.count("setp.eq.and.u32 %__agp2, %__agr2, 1, %__agp2;") == n_acc
    loads = sum(1 for x in s if x[1].startswith("ld."))
    stores = n_acc - loads
    if policy == "trap":
        assert out.count("@!%__agp3 trap;") == n_acc
    else:
        assert "trap;" not in out
    if policy == "poison":
        assert out.count("selp.b64 %__agd5, %__agd0, %__agT3, %__agp3") == loads   # zero page
        assert out.count("@%__agp4 st.global") == stores                            # predicated
    if policy == "sink":
        assert out.count("selp.b64 %__agd5, %__agd0, %__agT4, %__agp3") == stores  # sink page
    assemble(out)


def test_remap_policy_emission():
    """REMAP_OR: each denied access re-checks address | mask (header offset 104) with
    logging off; loads fall back to the zero page, stores and atomics are predicated on
    either check, and a dropped atomic's destination is zeroed before the original
    predicate joins in."""
    out, rep = ag.agile_guard_instrument_ptx(STREAM, "remap")
    n = rep["guarded"]
    assert n == 28
    assert out.count("ld.global.u64 %__agd6, [%__agT7+104];") == n
    assert len(slow_paths(out)) == 2 * n and out.count(KEEP_IN_REGS) == n
    loads = len(re.findall(r"\bld\.global\.", STREAM))
    assert out.count("selp.b64 %__agd5, %__agd5, %__agT3, %__agp4") == loads
    assert out.count("@%__agp4 st.global") == n - loads
    assemble(out)
    body = """
    setp.ne.u64 %p1, %rd1, 0;
    @%p1 atom.global.add.u32 %r1, [%rd1], 1;
    """
    out, _ = ag.agile_guard_instrument_ptx(kernel(body), "remap")
    zero, join = out.index("@!%__agp4 mov.b32 %r1, 0;"), out.index("and.pred %__agp4, %__agp4, %p1;")
    assert zero < join and "@%__agp4 atom.global.add.u32 %r1, [%__agd5], 1;" in out
    assemble(out)


def test_aperture_mode_emission():
    """With apertures the pass compiles the aperture rule into the module: the inline test
    is the apertures' hull (two compares and a wrap check, no table loads), the check
    function compares against each aperture as a constant, and the module carries its own
    zero and sink pages."""
    import agile_synth as syn
    ap = syn.table1_protected()
    aps = (ap.base, ap.size, ap.kind, ap.ident)
    out, rep = ag.agile_guard_instrument_ptx(STREAM, "poison", apertures=aps)
    assert rep["guarded"] == 28
    assert "__agile_aperture_mode = 1" in out and "__agile_zero_page[64]" in out
    assert "[__agile_guard_table];" not in out.split(".entry", 1)[1]   # no table in the kernels
    assert "%__agT7+136" not in out                                     # no class-map test
    assert out.count("setp.ge.u64 %__agp1, %__agd0, 0xf8000000000;") == 28      # hull end
    assert out.count("setp.le.u64 %__agp0, %__agd1, 0xf0000000000;") == 28      # hull start
    assert out.count("setp.lt.u64 %__agq1, %__agt0, 0xf1000000000;") == 28       # MMIO aperture
    assert out.count("selp.u32 %__ags2, 2, %__ags2, %__agq1;") == 28
    assert out.count("selp.u32 %__ags2, 1, %__ags2, %__agq1;") == 28
    assemble(out)
    for policy in ("sink", "report", "trap"):
        assemble(ag.agile_guard_instrument_ptx(STREAM, policy, apertures=aps)[0])


@pytest.mark.parametrize("bad,code", [
    ("remap", -1),
    ("sets", None),
])
def test_aperture_mode_refusals(bad, code):
    import agile_synth as syn
    ap = syn.table1_protected()
    if bad == "remap":
        with pytest.raises(ag.AgileError) as e:
            ag.agile_guard_instrument_ptx(STREAM, "remap", apertures=(ap.base, ap.size, ap.kind, ap.ident))
        assert e.value.code == code
        return
    cases = [
        (syn._ranges([0x1000] * 5, [16] * 5, [2] * 5, [1] * 5), -11),
        (syn._ranges([0x1000], [16], [syn.KIND_USER], [1]), -5),
        (syn._ranges([0x1000, 0x1008], [16, 16], [2, 2], [1, 2]), -2),
    ]
    for r, c in cases:
        with pytest.raises(ag.AgileError) as e:
            ag.agile_guard_instrument_ptx(STREAM, "poison", apertures=(r.base, r.size, r.kind, r.ident))
        assert e.value.code == c


def test_skip_list_leaves_trusted_functions_alone():
    out, rep = ag.agile_guard_instrument_ptx(STREAM, "poison", skip=["agile_ptx_copy"])
    assert rep["guarded"] == 20 and rep["skipped"] == 8 and rep["functions"] == 3
    body = out[out.index(".entry agile_ptx_copy"):out.index(".entry agile_ptx_scale")]
    assert "agile guard" not in body and "__agT" not in body
    assemble(out)


def test_violations_merged_in_registers_only_where_every_exit_is_seen():
    """Entry functions keep their count and smallest record in registers and merge them
    before each ret and exit (predicated like it) and at the body's end. A .func keeps
    merging each violation at once. When some .func can exit the thread, or under TRAP,
    no function keeps registers."""
    body = """
    ld.global.f32 %f1, [%rd1];
    setp.eq.f32 %p1, %f1, 0f00000000;
    @%p1 ret;
    @!%p1 exit;
    """
    out, _ = ag.agile_guard_instrument_ptx(kernel(body), "poison")
    assert out.count(KEEP_IN_REGS) == 1 and MERGE_AT_ONCE not in out
    assert "@%p1 call __agile_guard_flush" in out and "@!%p1 call __agile_guard_flush" in out
    assert out.count("call __agile_guard_flush, (__agfc, __agfk, __agfi);") == 4
    assert out.index("@%p1 call __agile_guard_flush") < out.index("@%p1 ret;")
    assemble(out)
    helper = HDR + """
.func helper(.param .b64 q)
{
    .reg .b64 %rd<2>;
    .reg .f32 %f<2>;
    ld.param.b64 %rd1, [q];
    ld.global.f32 %f1, [%rd1];
    ret;
}
.visible .entry k(.param .u64 p0)
{
    .reg .b64 %rd<2>;
    .reg .f32 %f<2>;
    ld.param.u64 %rd1, [p0];
    st.global.f32 [%rd1], %f1;
    ret;
}
"""
    out, rep = ag.agile_guard_instrument_ptx(helper, "poison")
    assert rep["guarded"] == 2
    assert out.count(MERGE_AT_ONCE) == 1 and out.count(KEEP_IN_REGS) == 1
    assemble(out)
    exiting = helper.replace("    ld.global.f32 %f1, [%rd1];\n    ret;", "    ld.global.f32 %f1, [%rd1];\n    exit;")
    assert exiting != helper
    out, _ = ag.agile_guard_instrument_ptx(exiting, "poison")
    assert out.count(MERGE_AT_ONCE) == 2 and KEEP_IN_REGS not in out
    assert "call __agile_guard_flush" not in out
    assemble(out)
    out, _ = ag.agile_guard_instrument_ptx(kernel(body), "trap")
    assert KEEP_IN_REGS not in out and "call __agile_guard_flush" not in out
    assemble(out)


def test_generic_and_other_spaces():
    body = """
    ld.f32 %f1, [%rd1];
    st.f32 [%rd1+8], %f1;
    ld.shared.f32 %f2, [%rd1];
    ld.local.f32 %f3, [%rd1];
    ld.const.f32 %f4, [%rd1];
    atom.add.u32 %r1, [%rd1+-4], 1;
    """
    regs = ".reg .b64 %rd<8>;\n.reg .f32 %f<8>;\n.reg .b32 %r<8>;"
    out, rep = ag.agile_guard_instrument_ptx(kernel(body, regs), "poison")
    assert rep["guarded"] == 3 and rep["generic_guarded"] == 3
    assert out.count("isspacep.global %__agp2, %__agd0") == 3
    assert "add.s64 %__agd0, %rd1, 8;" in out and "add.s64 %__agd0, %rd1, -4;" in out
    assert "ld.shared.f32 %f2, [%rd1];" in out and "ld.local.f32 %f3, [%rd1];" in out
    assert "@!%__agp3 mov.b32 %r1, 0;" in out                 # denied atom reads 0
    assemble(out)


def test_predicated_accesses_combine_predicates():
    body = """
    setp.ne.u64 %p1, %rd1, 0;
    @%p1 st.global.f32 [%rd1], %f1;
    @!%p1 ld.global.f32 %f2, [%rd1+4];
    @%p1 red.global.add.u32 [%rd1], %r1;
    """
    out, rep = ag.agile_guard_instrument_ptx(kernel(body), "poison")
    assert rep["guarded"] == 3
    assert "and.pred %__agp4, %__agp3, %p1;" in out
    assert "@%__agp4 st.global.f32 [%__agd0], %f1;" in out
    assert "@!%p1 ld.global.f32 %f2, [%__agd5];" in out
    assert "or.pred %__agp1, %__agp1, %p1;" in out            # @!%p1: slow path only if p1 false
    assemble(out)


def test_vector_symbol_and_wide_accesses():
    body = """
    ld.global.nc.v2.u64 {%rd2, %rd3}, [%rd1];
    ld.global.v8.f32 {%f0, %f1, %f2, %f3, %f4, %f5, %f6, %f7}, [%rd1+32];
    st.global.b128 [%rd1], %q1;
    atom.global.cas.b32 %r1, [%rd1], %r2, %r3;
    ld.global.u32 %r4, [gv+4];
    """
    regs = ".reg .b64 %rd<8>;\n.reg .f32 %f<8>;\n.reg .b32 %r<8>;\n.reg .b128 %q<2>;"
    src = HDR + ".global .align 8 .u32 gv[4];\n" + kernel(body, regs)[len(HDR):]
    out, rep = ag.agile_guard_instrument_ptx(src, "sink")
    assert [int(x[2]) for x in sites(out)] == [16, 32, 16, 4, 4]
    assert "mov.u64 %__agd0, gv;" in out
    assemble(out)


@pytest.mark.parametrize("bad,code", [
    ("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%rd1], [%rd2], 16, [%rd3];", -9),
    ("cp.async.ca.shared.global [%rd1], [%rd2], 16;", -9),
    ("st.async.b32 [%rd1], %r1, [%rd2];", -9),
    ("multimem.ld_reduce.relaxed.sys.global.add.f32 %f1, [%rd1];", -9),
    ("discard.global.L2 [%rd1], 128;", -9),
])
def test_uncoverable_forms_rejected(bad, code):
    with pytest.raises(ag.AgileError) as e:
        ag.agile_guard_instrument_ptx(kernel(bad), "poison")
    assert e.value.code == code


def test_rejects_guard_names_and_bad_modules():
    out, _ = ag.agile_guard_instrument_ptx(STREAM, "poison")
    with pytest.raises(ag.AgileError) as e:            # output cannot be fed back in
        ag.agile_guard_instrument_ptx(out, "poison")
    assert e.value.code == -9
    with pytest.raises(ag.AgileError) as e:            # forging the table pointer
        ag.agile_guard_instrument_ptx(HDR + ".global .u64 __agile_guard_table;\n", "poison")
    assert e.value.code == -9
    with pytest.raises(ag.AgileError) as e:
        ag.agile_guard_instrument_ptx(".version 9.0\n.target sm_103a\n.address_size 32\n", "poison")
    assert e.value.code == -9
    with pytest.raises(ag.AgileError) as e:            # unbalanced body
        ag.agile_guard_instrument_ptx(kernel("ld.global.f32 %f1, [%rd1];")[:-3], "poison")
    assert e.value.code == -8


def test_labels_comments_and_scopes():
    body = """
    // a comment with ld.global.f32 in it: not an access
    /* block comment st.global.f32 [%rd1], %f1; */
$L1:
    {
    .reg .f32 %ff;
    ld.global.f32 %ff, [%rd1];   // inside a scope
    }
$L2: ld.global.f32 %f1, [%rd1+4];
    """
    out, rep = ag.agile_guard_instrument_ptx(kernel(body), "report")
    assert rep["guarded"] == 2
    assert "$L1:" in out and "$L2:" in out
    assemble(out)


def _random_body(rng, n_stmt):
    """Random statements over global, generic, shared, local and const accesses, some
    predicated, with vector forms and offsets. Returns (body, n_global, n_generic)."""
    loads = [("u8", "%rs1"), ("u16", "%rs2"), ("u32", "%r1"), ("u64", "%rd5"), ("f32", "%f1"),
             ("v2.f32", "{%f2, %f3}"), ("v4.f32", "{%f4, %f5, %f6, %f7}"), ("v2.u64", "{%rd6, %rd7}")]
    stores = [("u8", "%rs1"), ("u32", "%r1"), ("f32", "%f1"), ("v2.f32", "{%f2, %f3}"),
              ("v4.f32", "{%f4, %f5, %f6, %f7}"), ("u64", "%rd5")]
    lines, ng, ngen = [], 0, 0
    for _ in range(n_stmt):
        pred = rng.choice(["", "", "@%p1 ", "@!%p1 "])
        off = rng.choice(["", "+8", "+-16", "+4096"])
        base = rng.choice(["%rd1", "%rd2"])
        kind = rng.randrange(9)
        if kind == 0:
            t, d = rng.choice(loads)
            nc = rng.choice(["", ".nc"])
            lines.append(f"{pred}ld.global{nc}.{t} {d}, [{base}{off}];"); ng += 1
        elif kind == 1:
            t, sv = rng.choice(stores)
            lines.append(f"{pred}st.global.{t} [{base}{off}], {sv};"); ng += 1
        elif kind == 2:
            lines.append(f"{pred}atom.global.add.u32 %r2, [{base}{off}], 1;"); ng += 1
        elif kind == 3:
            lines.append(f"{pred}red.global.add.u32 [{base}{off}], %r1;"); ng += 1
        elif kind == 4:
            lines.append(f"{pred}ld.f32 %f1, [{base}{off}];"); ng += 1; ngen += 1
        elif kind == 5:
            lines.append(f"{pred}st.u32 [{base}{off}], %r1;"); ng += 1; ngen += 1
        elif kind == 6:
            lines.append(f"{pred}ld.shared.f32 %f1, [%r3];")
        elif kind == 7:
            lines.append(f"{pred}ld.local.u32 %r1, [%rd3];")
        else:
            lines.append("add.f32 %f1, %f1, %f2;")
    return "\n".join(lines), ng, ngen


RAND_REGS = (".reg .b64 %rd<8>;\n.reg .f32 %f<8>;\n.reg .b32 %r<4>;\n.reg .b16 %rs<3>;\n"
             ".reg .pred %p<2>;\nsetp.ne.u64 %p1, %rd1, 0;\nmov.u64 %rd2, %rd1;\nmov.u32 %r3, 0;\n"
             "mov.u64 %rd3, 0;")


@pytest.mark.parametrize("seed", range(6))
def test_random_kernels_every_global_access_guarded(seed):
    """Random mixes of access forms: the report counts exactly the global and generic
    accesses, each gets one site, other spaces stay untouched, and the output assembles
    for sm_103a under every policy and under the aperture rule."""
    import random
    import agile_synth as syn
    rng = random.Random(1000 + seed)
    body, ng, ngen = _random_body(rng, 40)
    src = kernel(body, RAND_REGS)
    ap = syn.table1_protected()
    variants = [(p, None) for p in ("poison", "sink", "report", "trap", "remap")]
    variants += [(p, (ap.base, ap.size, ap.kind, ap.ident)) for p in ("poison", "report")]
    for policy, aps in variants:
        out, rep = ag.agile_guard_instrument_ptx(src, policy, apertures=aps)
        assert rep["guarded"] == ng and rep["generic_guarded"] == ngen, (policy, rep)
        assert len(sites(out)) == ng
        assert out.count("ld.shared.f32 %f1, [%r3];") == body.count("ld.shared.f32 %f1, [%r3];")
        assemble(out)
