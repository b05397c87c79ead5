"""Oracle for the kernel memory guard -- TEST INFRASTRUCTURE ONLY.

A ctypes front for ``agile_oracle.c`` (plain single-threaded C, compiled here with gcc).
Only the tests, the smoke check and the benchmark's CPU-baseline leg may import this
package; the product library never does, and this package imports nothing from it.

Every function cites the passage of the paper it follows; the classification rule is
stated in full at the top of ``agile_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "agile_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

VERDICT_NAMES = ["ALLOW", "PROTECTED", "MMIO", "STRADDLE", "UNMAPPED", "INVALID", "NOT_EXACT"]
NO_RANGE = 0xFFFFFFFF
POLICY = {"poison": 0, "sink": 1, "report": 2, "remap": 4}
RULES = {"table": 0, "aperture": 1}
STREAM_OPS = {"copy": 0, "scale": 1, "triad": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                        "-fno-fast-math", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Log(ctypes.Structure):
    _fields_ = [("key", ctypes.c_uint64), ("addr", ctypes.c_uint64), ("width", ctypes.c_uint32),
                ("verdict", ctypes.c_uint32), ("site", ctypes.c_uint32),
                ("range_id", ctypes.c_uint32), ("count", ctypes.c_uint64)]


@dataclass(frozen=True)
class Log:
    """First violation (smallest key) and the number of violations; count 0 = empty."""
    key: int
    addr: int
    width: int
    verdict: int
    site: int
    range_id: int
    count: int

    @staticmethod
    def _of(c: _Log) -> "Log":
        if c.count == 0:
            return Log(0, 0, 0, 0, 0, NO_RANGE, 0)
        return Log(c.key, c.addr, c.width, c.verdict, c.site, c.range_id, c.count)


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _table(r):
    base = np.ascontiguousarray(r.base, dtype=np.uint64)
    size = np.ascontiguousarray(r.size, dtype=np.uint64)
    kind = np.ascontiguousarray(r.kind, dtype=np.uint32)
    ident = np.ascontiguousarray(r.ident, dtype=np.uint32)
    return base, size, kind, ident


def table_check(r) -> int:
    """0 if the ranges form a legal table, else why not (1 zero size, 2 end beyond
    2**64-1, 3 two ranges share a byte, 4 unknown kind). Sec. V-C: each allocation is a
    (base, size) record; the three kinds are Table I's."""
    base, size, kind, _ = _table(r)
    f = _L().orc_table_check
    f.restype = ctypes.c_int
    return f(ctypes.c_size_t(len(base)), _p(base), _p(size), _p(kind))


def check_batch(r, addr: np.ndarray, width: np.ndarray, method: str = "linear"):
    """Verdict and deciding range id per (address, width) and the violation log
    (Sec. IV-E classification, Sec. V-E logging; first fault = smallest access index).
    method: 'linear' (the definition) or 'sorted' (binary search, pinned to linear)."""
    base, size, kind, ident = _table(r)
    addr = np.ascontiguousarray(addr, dtype=np.uint64)
    width = np.ascontiguousarray(width, dtype=np.uint8)
    m = len(addr)
    verdict = np.empty(m, dtype=np.uint8)
    rid = np.empty(m, dtype=np.uint32)
    log = _Log()
    _L().orc_check_batch(ctypes.c_size_t(len(base)), _p(base), _p(size), _p(kind), _p(ident),
                         ctypes.c_size_t(m), _p(addr), _p(width), _p(verdict), _p(rid),
                         ctypes.byref(log), ctypes.c_int(0 if method == "linear" else 1))
    return verdict, rid, Log._of(log)


def aperture_batch(apertures, addr: np.ndarray, width: np.ndarray):
    """Aperture rule (Table I, Sec. V-E): deny only accesses that share a byte with a
    protected or MMIO aperture (MMIO first, lowest base), INVALID as in check_batch,
    everything else allowed. Returns (verdict, range id, Log); key = access index."""
    base, size, kind, ident = _table(apertures)
    addr = np.ascontiguousarray(addr, dtype=np.uint64)
    width = np.ascontiguousarray(width, dtype=np.uint8)
    m = len(addr)
    verdict = np.empty(m, dtype=np.uint8)
    rid = np.empty(m, dtype=np.uint32)
    log = _Log()
    _L().orc_aperture_batch(ctypes.c_size_t(len(base)), _p(base), _p(size), _p(kind), _p(ident),
                            ctypes.c_size_t(m), _p(addr), _p(width), _p(verdict), _p(rid),
                            ctypes.byref(log))
    return verdict, rid, Log._of(log)


def validate(r, ptr: np.ndarray, nbytes: np.ndarray):
    """API-time pointer validation, Sec. IV-E and V-C: a (pointer, byte count) passes
    only when the whole byte range lies inside one live user allocation."""
    base, size, kind, ident = _table(r)
    ptr = np.ascontiguousarray(ptr, dtype=np.uint64)
    nbytes = np.ascontiguousarray(nbytes, dtype=np.uint64)
    m = len(ptr)
    verdict = np.empty(m, dtype=np.uint8)
    rid = np.empty(m, dtype=np.uint32)
    _L().orc_validate(ctypes.c_size_t(len(base)), _p(base), _p(size), _p(kind), _p(ident),
                      ctypes.c_size_t(m), _p(ptr), _p(nbytes), _p(verdict), _p(rid))
    return verdict, rid


def validate_exact(r, ptr: np.ndarray, nbytes: np.ndarray):
    """DMA registration, Sec. V-C: accepted only for an exact live user allocation;
    a byte range strictly inside one is NOT_EXACT (6); otherwise the ordinary verdict."""
    base, size, kind, ident = _table(r)
    ptr = np.ascontiguousarray(ptr, dtype=np.uint64)
    nbytes = np.ascontiguousarray(nbytes, dtype=np.uint64)
    m = len(ptr)
    verdict = np.empty(m, dtype=np.uint8)
    rid = np.empty(m, dtype=np.uint32)
    _L().orc_validate_exact(ctypes.c_size_t(len(base)), _p(base), _p(size), _p(kind), _p(ident),
                            ctypes.c_size_t(m), _p(ptr), _p(nbytes), _p(verdict), _p(rid))
    return verdict, rid


def stream(op: str, r, va: dict, b: np.ndarray, c: np.ndarray | None, a0: np.ndarray,
           s: float = 3.0, policy: str = "poison", rule: str = "table"):
    """Guarded copy / scale / triad (Sec. V-E guard and policies; access order stated in
    agile_oracle.c). va: {'a','b','c'} -> guarded-space addresses. rule 'aperture' checks
    against the ranges r as apertures (Table I rule). Returns (a, log)."""
    base, size, kind, ident = _table(r)
    n = len(b)
    b = np.ascontiguousarray(b, dtype=np.float32)
    c = np.ascontiguousarray(c if c is not None else np.zeros(n, np.float32), dtype=np.float32)
    a = np.array(a0, dtype=np.float32, copy=True)
    log = _Log()
    _L().orc_stream(ctypes.c_int(STREAM_OPS[op]), ctypes.c_size_t(n), ctypes.c_uint64(va["a"]),
                    ctypes.c_uint64(va["b"]), ctypes.c_uint64(va.get("c", 0)), ctypes.c_float(s),
                    _p(b), _p(c), _p(a), ctypes.c_int(POLICY[policy]),
                    ctypes.c_int(RULES[rule]),
                    ctypes.c_size_t(len(base)), _p(base), _p(size), _p(kind), _p(ident),
                    ctypes.byref(log))
    return a, Log._of(log)


def stream_plain(op: str, b: np.ndarray, c: np.ndarray | None, s: float = 3.0) -> np.ndarray:
    """Unguarded copy / scale / triad; triad is one fused multiply-add (fmaf)."""
    n = len(b)
    b = np.ascontiguousarray(b, dtype=np.float32)
    c = np.ascontiguousarray(c if c is not None else np.zeros(n, np.float32), dtype=np.float32)
    a = np.empty(n, dtype=np.float32)
    _L().orc_stream_plain(ctypes.c_int(STREAM_OPS[op]), ctypes.c_size_t(n), ctypes.c_float(s),
                          _p(b), _p(c), _p(a))
    return a


IRREGULAR = {"gather": 0, "scatter": 1, "hist": 2}


def irregular(kind: str, r, arena: np.ndarray, arena_va: int, va: dict, n: int,
              policy: str = "poison", remap: int = 0, rule: str = "table"):
    """Guarded gather / scatter / histogram over an arena copy (Sec. V-E guard and
    policies; access order stated in agile_oracle.c). `arena` (uint8) is updated in
    place; va: {'idx', 't', 'out'} guarded-space addresses; remap is the REMAP_OR mask.
    Returns the Log."""
    base, size, kind_, ident = _table(r)
    assert arena.dtype == np.uint8 and arena.flags.c_contiguous
    log = _Log()
    f = _L().orc_irregular
    f.restype = ctypes.c_int
    rc = f(ctypes.c_int(IRREGULAR[kind]), ctypes.c_size_t(n), ctypes.c_uint64(arena_va),
           _p(arena), ctypes.c_size_t(len(arena)), ctypes.c_uint64(va["idx"]),
           ctypes.c_uint64(va["t"]), ctypes.c_uint64(va.get("out", 0)),
           ctypes.c_int(POLICY[policy]), ctypes.c_uint64(remap), ctypes.c_int(RULES[rule]),
           ctypes.c_size_t(len(base)),
           _p(base), _p(size), _p(kind_), _p(ident), ctypes.byref(log))
    if rc != 0:
        raise ValueError("an access that is carried out falls outside the arena")
    return Log._of(log)
