"""ctypes binding of the C ABI in ``include/agile_guard.h`` (same names, same arguments).

Host arrays are numpy; device buffers are anything with ``data_ptr()`` (torch tensors)
or a raw integer address; streams are ``torch.cuda.Stream`` objects, raw cudaStream_t
integers, or None for the legacy default stream.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libagileguard.so")

LOG_BYTES = 64
LIST_HEADER_BYTES = 16
LIST_ENTRY_BYTES = 32


def list_bytes(capacity: int) -> int:
    """Device bytes of a bounded violation list of `capacity` entries (AGILE_LIST_BYTES)."""
    return LIST_HEADER_BYTES + capacity * LIST_ENTRY_BYTES
NO_RANGE = 0xFFFFFFFF
VERDICTS = ["ALLOW", "PROTECTED", "MMIO", "STRADDLE", "UNMAPPED", "INVALID", "NOT_EXACT"]
KINDS = {"user": 0, "protected": 1, "mmio": 2}
POLICIES = {"poison": 0, "sink": 1, "report": 2, "trap": 3, "remap": 4}
OPS = {"copy": 0, "scale": 1, "triad": 2}
IRREGULAR = {"gather": 0, "scatter": 1, "hist": 2}
WORK = {"copy": 0, "scale": 1, "triad": 2, "gather": 3, "scatter": 4, "hist": 5}


class AgileError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {agile_strerror(code)} ({code})")


class _Range(ctypes.Structure):
    _fields_ = [("base", ctypes.c_uint64), ("size", ctypes.c_uint64),
                ("kind", ctypes.c_uint32), ("id", ctypes.c_uint32)]


class _DevTable(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("npages", ctypes.c_uint64),
                ("log2_page", ctypes.c_uint32), ("n", ctypes.c_uint32),
                ("page", ctypes.c_void_p), ("base", ctypes.c_void_p), ("end", ctypes.c_void_p),
                ("kind", ctypes.c_void_p), ("id", ctypes.c_void_p),
                ("zero_page", ctypes.c_void_p), ("sink_page", ctypes.c_void_p),
                ("bytes", ctypes.c_uint64), ("search_steps", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("crange", ctypes.c_void_p),
                ("remap_or", ctypes.c_uint64), ("ubits", ctypes.c_void_p),
                ("ubits_log2", ctypes.c_uint32), ("ubits_n", ctypes.c_uint32),
                ("cmap", ctypes.c_void_p), ("cmap_log2", ctypes.c_uint32),
                ("cmap_n", ctypes.c_uint32), ("cdesc", ctypes.c_void_p),
                ("cdesc_log2", ctypes.c_uint32), ("cdesc_k1", ctypes.c_uint32),
                ("cdesc_k2", ctypes.c_uint32), ("cdesc_reserved", ctypes.c_uint32)]


class _Record(ctypes.Structure):
    _fields_ = [("key", ctypes.c_uint64), ("addr", ctypes.c_uint64), ("width", ctypes.c_uint32),
                ("verdict", ctypes.c_uint32), ("site", ctypes.c_uint32),
                ("range_id", ctypes.c_uint32), ("client", ctypes.c_uint32),
                ("status", ctypes.c_uint32), ("count", ctypes.c_uint64)]


class Work(ctypes.Structure):
    """agile_work_t: one client's guarded kernel inside a batch."""
    _fields_ = [("op", ctypes.c_uint32), ("policy", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("table", ctypes.c_void_p), ("log", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("in0", ctypes.c_void_p), ("in1", ctypes.c_void_p), ("s", ctypes.c_float),
                ("client", ctypes.c_uint32)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_uint32), ("span_checks", ctypes.c_uint32),
                ("blocks_per_sm", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("config", BatchConfig), ("variant", ctypes.c_uint32), ("cached", ctypes.c_uint32),
                ("ms", ctypes.c_float)]


class Request(ctypes.Structure):
    """agile_request_t."""
    _fields_ = [("tag", ctypes.c_uint64), ("client", ctypes.c_uint32), ("nargs", ctypes.c_uint32),
                ("arg_ptr", ctypes.c_uint64 * 16), ("arg_bytes", ctypes.c_uint64 * 16),
                ("work", Work), ("mem_bytes", ctypes.c_uint64), ("excl", ctypes.c_uint64),
                ("arrival_ns", ctypes.c_uint64)]


class Completion(ctypes.Structure):
    """agile_completion_t."""
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("bad_arg", ctypes.c_uint32),
                ("verdict", ctypes.c_uint32), ("launch", ctypes.c_uint32),
                ("arrival_ns", ctypes.c_uint64), ("admit_ns", ctypes.c_uint64),
                ("done_ns", ctypes.c_uint64), ("seen_ns", ctypes.c_uint64),
                ("queued_ns", ctypes.c_uint64)]


class WorkerConfig(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("max_inflight", ctypes.c_uint32), ("tile", ctypes.c_uint32),
                ("continuous", ctypes.c_uint32)]


class _InstrOpts(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int), ("skip", ctypes.POINTER(ctypes.c_char_p)),
                ("nskip", ctypes.c_size_t), ("apertures", ctypes.c_void_p),
                ("napertures", ctypes.c_size_t)]


class _InstrReport(ctypes.Structure):
    _fields_ = [("functions", ctypes.c_uint32), ("guarded", ctypes.c_uint32),
                ("generic_guarded", ctypes.c_uint32), ("skipped", ctypes.c_uint32)]


_P = ctypes.c_void_p
_SIG = {
    "agile_guard_table_build": (ctypes.c_int, [_P, ctypes.c_size_t, ctypes.c_uint32, _P]),
    "agile_guard_table_device_bytes": (ctypes.c_int, [_P, _P]),
    "agile_guard_table_set_remap": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "agile_guard_table_geometry": (ctypes.c_int, [_P, _P, _P]),
    "agile_guard_table_upload": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P, _P]),
    "agile_guard_table_image": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "agile_guard_table_destroy": (None, [_P]),
    "agile_validate_args": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t, _P, _P]),
    "agile_validate_dma": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t, _P, _P]),
    "agile_violation_log_init": (ctypes.c_int, [_P, ctypes.c_uint32, _P]),
    "agile_violation_log_read": (ctypes.c_int, [_P, _P, _P]),
    "agile_violation_list_attach": (ctypes.c_int, [_P, _P, ctypes.c_uint32, _P]),
    "agile_violation_list_read": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t, _P, _P, _P]),
    "agile_guard_check_batch": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t, _P, _P, _P]),
    "agile_aperture_check_batch": (ctypes.c_int, [_P, ctypes.c_size_t, _P, _P, ctypes.c_size_t,
                                                  _P, _P, _P]),
    "agile_stream_launch": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, ctypes.c_size_t,
                                           ctypes.c_float, ctypes.c_int, _P, _P]),
    "agile_stream_launch_shape": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, ctypes.c_size_t,
                                                 ctypes.c_float, ctypes.c_int, _P, ctypes.c_int,
                                                 ctypes.c_int, _P]),
    "agile_irregular_launch": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, ctypes.c_size_t,
                                              ctypes.c_int, _P, _P]),
    "agile_irregular_launch_fastpath": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, ctypes.c_size_t,
                                                       ctypes.c_int, _P, ctypes.c_int, _P]),
    "agile_stream_launch_host": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, _P, _P, _P,
                                                ctypes.c_size_t, ctypes.c_float, ctypes.c_int, _P,
                                                ctypes.c_size_t, _P]),
    "agile_batch_device_bytes": (ctypes.c_size_t, [ctypes.c_size_t]),
    "agile_batch_upload": (ctypes.c_int, [_P, ctypes.c_size_t, ctypes.c_uint32, _P, ctypes.c_size_t, _P]),
    "agile_batch_launch": (ctypes.c_int, [_P, ctypes.c_size_t, _P, _P]),
    "agile_batch_graph_create": (ctypes.c_int, [_P, ctypes.c_size_t, _P, _P]),
    "agile_graph_launch": (ctypes.c_int, [_P, _P]),
    "agile_graph_destroy": (None, [_P]),
    "agile_batch_launch_static": (ctypes.c_int, [_P, ctypes.c_size_t, ctypes.c_uint32, _P, _P]),
    "agile_batch_autotune": (ctypes.c_int, [_P, ctypes.c_size_t, ctypes.c_size_t, _P, ctypes.c_size_t,
                                            _P, ctypes.c_size_t, ctypes.c_int, ctypes.c_char_p, _P, _P]),
    "agile_worker_device_bytes": (ctypes.c_size_t, [_P]),
    "agile_worker_create": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_size_t, _P, ctypes.c_size_t, _P]),
    "agile_worker_submit": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "agile_worker_start": (ctypes.c_int, [_P]),
    "agile_worker_poll": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P, ctypes.c_uint32]),
    "agile_worker_clock": (ctypes.c_int, [_P, _P, _P, _P]),
    "agile_worker_destroy": (None, [_P]),
    "agile_guard_instrument_ptx": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_size_t, _P, _P, _P, _P]),
    "agile_module_load": (ctypes.c_int, [ctypes.c_char_p, _P]),
    "agile_module_bind": (ctypes.c_int, [_P, _P, _P, _P]),
    "agile_module_launch": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_uint32, ctypes.c_uint32,
                                           _P, _P]),
    "agile_module_unload": (None, [_P]),
    "agile_selftest_bounded_waits": (ctypes.c_int, [_P, _P, ctypes.c_uint32, _P, _P]),
    "agile_free": (None, [_P]),
    "agile_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "agile_version": (ctypes.c_uint32, []),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library. Raises if it is missing: there is no fallback path."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise ImportError(f"{library_path} is missing: build it with "
                              "`python -m paper_2606_06697_b300.build`")
        L = ctypes.CDLL(library_path)
        for name, (res, args) in _SIG.items():
            try:
                f = getattr(L, name)
            except AttributeError:
                continue            # calling it raises AttributeError: never a silent path
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, where: str, ok=(0,)) -> int:
    if rc not in ok:
        raise AgileError(rc, where)
    return rc


def _dptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _hptr(x) -> int | None:
    """Host buffer address: None, an int, a numpy array or a CPU tensor."""
    if x is None or isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def agile_strerror(code: int) -> str:
    return lib().agile_strerror(code).decode()


def agile_version() -> int:
    return lib().agile_version()


def agile_free(p) -> None:
    lib().agile_free(p)


# ---------------------------------------------------------------- table


class DevTable:
    """An uploaded table: the device view plus a reference to its buffer."""

    def __init__(self, view: _DevTable, buf):
        self.view = view
        self.buf = buf

    @property
    def ref(self):
        return ctypes.byref(self.view)

    @property
    def address(self) -> int:
        return _dptr(self.buf)


class Table:
    """Host table object; frees itself."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.agile_guard_table_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    @property
    def handle(self):
        return self._h

    def device_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().agile_guard_table_device_bytes(self._h, ctypes.byref(n)),
               "agile_guard_table_device_bytes")
        return n.value

    def geometry(self):
        lg = ctypes.c_uint32()
        npg = ctypes.c_uint64()
        _check(lib().agile_guard_table_geometry(self._h, ctypes.byref(lg), ctypes.byref(npg)),
               "agile_guard_table_geometry")
        return lg.value, npg.value

    def set_remap(self, mask: int) -> None:
        """agile_guard_table_set_remap: the REMAP_OR mask for later uploads."""
        _check(lib().agile_guard_table_set_remap(self._h, mask), "agile_guard_table_set_remap")

    def upload(self, buf, stream=None) -> DevTable:
        """agile_guard_table_upload into `buf` (a uint8 CUDA tensor of >= device_bytes)."""
        v = _DevTable()
        nbytes = buf.numel() * buf.element_size() if hasattr(buf, "numel") else self.device_bytes()
        _check(lib().agile_guard_table_upload(self._h, _dptr(buf), nbytes, _stream(stream),
                                              ctypes.byref(v)), "agile_guard_table_upload")
        return DevTable(v, buf)

    def image(self):
        """agile_guard_table_image into a fresh 256-byte aligned host buffer: returns the
        view (pointers into the buffer), the buffer's address and the image as a uint8
        numpy array (which keeps the buffer alive)."""
        nbytes = self.device_bytes()
        raw = np.zeros(nbytes + 256, dtype=np.uint8)
        off = (-raw.ctypes.data) % 256
        img = raw[off:off + nbytes]
        v = _DevTable()
        _check(lib().agile_guard_table_image(self._h, ctypes.c_void_p(img.ctypes.data), nbytes,
                                             ctypes.byref(v)), "agile_guard_table_image")
        return v, img.ctypes.data, img


def _range_array(base, size, kind, ident):
    base = _np(base, np.uint64)
    n = len(base)
    arr = (_Range * max(n, 1))()
    raw = np.frombuffer(arr, dtype=np.dtype([("base", "<u8"), ("size", "<u8"),
                                             ("kind", "<u4"), ("id", "<u4")]), count=max(n, 1))
    if n:
        raw["base"] = base
        raw["size"] = _np(size, np.uint64)
        raw["kind"] = _np(kind, np.uint32)
        raw["id"] = _np(ident, np.uint32)
    return arr, n


def agile_guard_table_build(base, size, kind, ident, log2_page: int = 21) -> Table:
    """Build a table from parallel arrays (any order)."""
    arr, n = _range_array(base, size, kind, ident)
    out = ctypes.c_void_p()
    _check(lib().agile_guard_table_build(arr, n, log2_page, ctypes.byref(out)),
           "agile_guard_table_build")
    return Table(out.value)


def agile_validate_args(table: Table, ptr, nbytes):
    """Returns (rc, verdict uint8[n], range_id uint32[n]); rc 0 or AGILE_VIOLATION."""
    ptr = _np(ptr, np.uint64)
    nbytes = _np(nbytes, np.uint64)
    v = np.empty(len(ptr), np.uint8)
    rid = np.empty(len(ptr), np.uint32)
    rc = _check(lib().agile_validate_args(table.handle, ptr.ctypes.data, nbytes.ctypes.data,
                                          len(ptr), v.ctypes.data, rid.ctypes.data),
                "agile_validate_args", ok=(0, 1))
    return rc, v, rid


def agile_validate_dma(table: Table, ptr, nbytes):
    """DMA registration check: (rc, verdict uint8[n], range_id uint32[n])."""
    ptr = _np(ptr, np.uint64)
    nbytes = _np(nbytes, np.uint64)
    v = np.empty(len(ptr), np.uint8)
    rid = np.empty(len(ptr), np.uint32)
    rc = _check(lib().agile_validate_dma(table.handle, ptr.ctypes.data, nbytes.ctypes.data,
                                         len(ptr), v.ctypes.data, rid.ctypes.data),
                "agile_validate_dma", ok=(0, 1))
    return rc, v, rid


# ---------------------------------------------------------------- log


@dataclass(frozen=True)
class ViolationRecord:
    key: int
    addr: int
    width: int
    verdict: int
    site: int
    range_id: int
    client: int
    status: int
    count: int


def agile_violation_log_init(d_log, client: int = 0, stream=None) -> None:
    _check(lib().agile_violation_log_init(_dptr(d_log), client, _stream(stream)),
           "agile_violation_log_init")


def agile_violation_log_read(d_log, stream=None):
    """Returns (rc, ViolationRecord); rc 0, AGILE_VIOLATION (1) or AGILE_ERR_TIMEOUT."""
    r = _Record()
    rc = _check(lib().agile_violation_log_read(_dptr(d_log), ctypes.byref(r), _stream(stream)),
                "agile_violation_log_read", ok=(0, 1, -10))
    return rc, ViolationRecord(r.key, r.addr, r.width, r.verdict, r.site, r.range_id, r.client,
                               r.status, r.count)


def agile_violation_list_attach(d_log, d_list, capacity: int, stream=None) -> None:
    """Attach a bounded violation list (d_list: >= list_bytes(capacity) device bytes) to an
    initialized log."""
    _check(lib().agile_violation_list_attach(_dptr(d_log), _dptr(d_list), capacity, _stream(stream)),
           "agile_violation_list_attach")


def agile_violation_list_read(d_log, d_list, max_entries: int | None = None, stream=None):
    """Returns (records, n_seen): the list's entries as ViolationRecords, in the order the
    GPU took their slots, and the violations recorded since the attach."""
    if max_entries is None:
        max_entries = (d_list.numel() * d_list.element_size() - LIST_HEADER_BYTES) // LIST_ENTRY_BYTES
    buf = (_Record * max(1, max_entries))()
    n_out = ctypes.c_size_t()
    n_seen = ctypes.c_uint64()
    _check(lib().agile_violation_list_read(_dptr(d_log), _dptr(d_list), buf, max_entries,
                                           ctypes.byref(n_out), ctypes.byref(n_seen), _stream(stream)),
           "agile_violation_list_read")
    recs = [ViolationRecord(r.key, r.addr, r.width, r.verdict, r.site, r.range_id, r.client,
                            r.status, r.count) for r in buf[:n_out.value]]
    return recs, n_seen.value


# ---------------------------------------------------------------- device checks


def agile_guard_check_batch(dev: DevTable, d_addr, d_width, n: int, d_verdict, d_log=None,
                            stream=None) -> None:
    _check(lib().agile_guard_check_batch(dev.ref, _dptr(d_addr), _dptr(d_width), n,
                                         _dptr(d_verdict), _dptr(d_log), _stream(stream)),
           "agile_guard_check_batch")


def agile_aperture_check_batch(apertures, d_addr, d_width, n: int, d_verdict, d_log=None,
                               stream=None) -> None:
    """apertures: (base, size, kind, ident) parallel arrays, at most AGILE_MAX_APERTURES."""
    arr, m = _range_array(*apertures)
    _check(lib().agile_aperture_check_batch(arr, m, _dptr(d_addr), _dptr(d_width), n,
                                            _dptr(d_verdict), _dptr(d_log), _stream(stream)),
           "agile_aperture_check_batch")


def agile_stream_launch(op: str, dev: DevTable | None, d_a, d_b, d_c, n: int, s: float = 3.0,
                        policy: str = "poison", d_log=None, stream=None) -> None:
    _check(lib().agile_stream_launch(OPS[op], dev.ref if dev is not None else None, _dptr(d_a),
                                     _dptr(d_b), _dptr(d_c), n, s, POLICIES[policy], _dptr(d_log),
                                     _stream(stream)), "agile_stream_launch")


def agile_stream_launch_shape(op: str, dev: DevTable | None, d_a, d_b, d_c, n: int, s: float,
                              policy: str, d_log, units: int, blocks_per_sm: int,
                              stream=None) -> None:
    _check(lib().agile_stream_launch_shape(OPS[op], dev.ref if dev is not None else None,
                                           _dptr(d_a), _dptr(d_b), _dptr(d_c), n, s,
                                           POLICIES[policy], _dptr(d_log), units, blocks_per_sm,
                                           _stream(stream)), "agile_stream_launch_shape")


def agile_stream_launch_host(op: str, dev: DevTable | None, d_a, d_b, d_c, h_a, h_b, h_c, n: int,
                             s: float = 3.0, policy: str = "poison", d_log=None,
                             chunk_elems: int = 0, stream=None) -> None:
    """h_*: host buffers (pinned CPU tensors, numpy arrays or addresses) or None."""
    _check(lib().agile_stream_launch_host(OPS[op], dev.ref if dev is not None else None,
                                          _dptr(d_a), _dptr(d_b), _dptr(d_c), _hptr(h_a),
                                          _hptr(h_b), _hptr(h_c), n, s, POLICIES[policy],
                                          _dptr(d_log), chunk_elems, _stream(stream)),
           "agile_stream_launch_host")


def agile_irregular_launch(kind: str, dev: DevTable | None, d_idx, d_base, d_out, n: int,
                           policy: str = "poison", d_log=None, stream=None) -> None:
    _check(lib().agile_irregular_launch(IRREGULAR[kind], dev.ref if dev is not None else None,
                                        _dptr(d_idx), _dptr(d_base), _dptr(d_out), n,
                                        POLICIES[policy], _dptr(d_log), _stream(stream)),
           "agile_irregular_launch")


FAST_PATHS = {"bitmap": 0, "match": 1}


def agile_irregular_launch_fastpath(kind: str, dev: DevTable | None, d_idx, d_base, d_out, n: int,
                                    policy: str = "poison", d_log=None, fast_path: str = "bitmap",
                                    stream=None) -> None:
    _check(lib().agile_irregular_launch_fastpath(IRREGULAR[kind], dev.ref if dev is not None else None,
                                                 _dptr(d_idx), _dptr(d_base), _dptr(d_out), n,
                                                 POLICIES[policy], _dptr(d_log),
                                                 FAST_PATHS[fast_path], _stream(stream)),
           "agile_irregular_launch_fastpath")


# ---------------------------------------------------------------- batched clients


def make_work(op: str, dev: DevTable | None, out, in0, in1, n: int, s: float = 3.0,
              policy: str = "poison", log=None, client: int = 0) -> Work:
    return Work(WORK[op], POLICIES[policy], n, dev.address if dev is not None else None,
                _dptr(log), _dptr(out), _dptr(in0), _dptr(in1), s, client)


def agile_batch_device_bytes(max_items: int) -> int:
    return lib().agile_batch_device_bytes(max_items)


def agile_batch_upload(items, tile: int, d_buf, stream=None) -> None:
    arr = (Work * len(items))(*items)
    nbytes = d_buf.numel() * d_buf.element_size() if hasattr(d_buf, "numel") else \
        agile_batch_device_bytes(len(items))
    _check(lib().agile_batch_upload(arr, len(items), tile, _dptr(d_buf), nbytes, _stream(stream)),
           "agile_batch_upload")


def agile_batch_launch(d_buf, n_items: int, tile: int, span_checks: bool = True,
                       blocks_per_sm: int = 2, stream=None) -> None:
    cfg = BatchConfig(tile, int(span_checks), blocks_per_sm, 0)
    _check(lib().agile_batch_launch(_dptr(d_buf), n_items, ctypes.byref(cfg), _stream(stream)),
           "agile_batch_launch")


BATCH_STATIC_MAX_ITEMS = 2048


def agile_batch_launch_static(items, tile: int, span_checks: bool = True, blocks_per_sm: int = 2,
                              stream=None) -> None:
    """agile_batch_launch without a device buffer from the caller: for callers that cannot
    allocate device memory (their budget is spoken for, they must avoid the implicit
    synchronization of an allocation, or their host gives them no allocator). The
    library's own fixed scratch array holds the work list; concurrent calls race on it."""
    arr = (Work * len(items))(*items)
    cfg = BatchConfig(tile, int(span_checks), blocks_per_sm, 0)
    _check(lib().agile_batch_launch_static(arr, len(items), tile, ctypes.byref(cfg), _stream(stream)),
           "agile_batch_launch_static")


class Graph:
    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    def launch(self, stream=None) -> None:
        _check(lib().agile_graph_launch(self._h, _stream(stream)), "agile_graph_launch")

    def destroy(self) -> None:
        if self._h.value:
            lib().agile_graph_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            if _lib is not None:
                self.destroy()
        except Exception:
            pass


def agile_batch_graph_create(d_buf, n_items: int, tile: int, span_checks: bool = True,
                             blocks_per_sm: int = 2) -> Graph:
    cfg = BatchConfig(tile, int(span_checks), blocks_per_sm, 0)
    out = ctypes.c_void_p()
    _check(lib().agile_batch_graph_create(_dptr(d_buf), n_items, ctypes.byref(cfg), ctypes.byref(out)),
           "agile_batch_graph_create")
    return Graph(out.value)


def agile_batch_autotune(variants, tiles, d_buf, reps: int = 3, cache_path: str | None = None,
                         stream=None) -> dict:
    """variants: list of equal-length work lists. Returns the winning configuration."""
    n_items = len(variants[0])
    flat = [w for v in variants for w in v]
    arr = (Work * len(flat))(*flat)
    tl = (ctypes.c_uint32 * len(tiles))(*tiles)
    best = BatchTuning()
    nbytes = d_buf.numel() * d_buf.element_size()
    _check(lib().agile_batch_autotune(arr, len(variants), n_items, tl, len(tiles), _dptr(d_buf),
                                      nbytes, reps, cache_path.encode() if cache_path else None,
                                      _stream(stream), ctypes.byref(best)), "agile_batch_autotune")
    c = best.config
    return {"tile": c.tile, "span_checks": bool(c.span_checks), "blocks_per_sm": c.blocks_per_sm,
            "variant": best.variant, "cached": bool(best.cached), "ms": best.ms}


# ---------------------------------------------------------------- serving worker


class Worker:
    """A native serving worker (agile_worker_*). Keeps references to what it uses."""

    def __init__(self, cfg: WorkerConfig, tables, devs, logs, d_buf):
        n = len(tables)
        self._keep = (tables, devs, logs, d_buf)
        ht = (ctypes.c_void_p * n)(*[t.handle.value for t in tables])
        self._views = [d.view for d in devs]
        dt = (ctypes.c_void_p * n)(*[ctypes.addressof(v) for v in self._views])
        dl = (ctypes.c_void_p * n)(*[_dptr(x) for x in logs])
        out = ctypes.c_void_p()
        nbytes = d_buf.numel() * d_buf.element_size()
        _check(lib().agile_worker_create(ctypes.byref(cfg), ht, dt, dl, n, _dptr(d_buf), nbytes,
                                         ctypes.byref(out)), "agile_worker_create")
        self._h = out

    def submit(self, reqs) -> None:
        arr = (Request * len(reqs))(*reqs)
        _check(lib().agile_worker_submit(self._h, arr, len(reqs)), "agile_worker_submit")

    def start(self) -> None:
        _check(lib().agile_worker_start(self._h), "agile_worker_start")

    def poll(self, cap: int = 4096, wait_ms: int = 50):
        arr = (Completion * cap)()
        got = ctypes.c_size_t()
        _check(lib().agile_worker_poll(self._h, arr, cap, ctypes.byref(got), wait_ms), "agile_worker_poll")
        return [arr[i] for i in range(got.value)]

    def clock(self):
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().agile_worker_clock(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "agile_worker_clock")
        return a.value, b.value, c.value

    def destroy(self) -> None:
        if self._h and self._h.value:
            lib().agile_worker_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            if _lib is not None:
                self.destroy()
        except Exception:
            pass


def agile_worker_device_bytes(cfg: WorkerConfig) -> int:
    return lib().agile_worker_device_bytes(ctypes.byref(cfg))


# ---------------------------------------------------------------- PTX guard pass


def agile_guard_instrument_ptx(ptx: str, policy: str = "poison", skip=(), apertures=None):
    """Returns (instrumented PTX text, report dict). apertures: (base, size, kind, ident)
    parallel arrays selecting the aperture rule, or None for the table rule."""
    names = [s.encode() for s in skip]
    arr = (ctypes.c_char_p * max(len(names), 1))(*names) if names else None
    ap_arr, n_ap = _range_array(*apertures) if apertures is not None else (None, 0)
    opts = _InstrOpts(POLICIES[policy], ctypes.cast(arr, ctypes.POINTER(ctypes.c_char_p))
                      if arr is not None else None, len(names),
                      ctypes.cast(ap_arr, ctypes.c_void_p) if n_ap else None, n_ap)
    out = ctypes.c_void_p()
    out_len = ctypes.c_size_t()
    rep = _InstrReport()
    data = ptx.encode()
    _check(lib().agile_guard_instrument_ptx(data, len(data), ctypes.byref(opts), ctypes.byref(out),
                                            ctypes.byref(out_len), ctypes.byref(rep)),
           "agile_guard_instrument_ptx")
    try:
        text = ctypes.string_at(out.value, out_len.value).decode()
    finally:
        lib().agile_free(out)
    return text, {"functions": rep.functions, "guarded": rep.guarded,
                  "generic_guarded": rep.generic_guarded, "skipped": rep.skipped}


class Module:
    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def unload(self):
        if self._h.value:
            lib().agile_module_unload(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            if _lib is not None:
                self.unload()
        except Exception:
            pass


def agile_module_unload(m: Module) -> None:
    m.unload()


def agile_module_load(ptx: str) -> Module:
    out = ctypes.c_void_p()
    _check(lib().agile_module_load(ptx.encode(), ctypes.byref(out)), "agile_module_load")
    return Module(out.value)


def agile_module_bind(m: Module, dev: DevTable | None, d_log=None, stream=None) -> None:
    """dev may be None for a module instrumented with apertures."""
    _check(lib().agile_module_bind(m.handle, dev.ref if dev is not None else None, _dptr(d_log),
                                   _stream(stream)), "agile_module_bind")


def agile_module_launch(m: Module, name: str, grid: int, block: int, args, stream=None) -> None:
    """args: list of ctypes scalars (c_uint64 for pointers, c_float, ...)."""
    arr = (ctypes.c_void_p * max(len(args), 1))(*[ctypes.cast(ctypes.pointer(a), ctypes.c_void_p)
                                                   for a in args])
    _check(lib().agile_module_launch(m.handle, name.encode(), grid, block, arr, _stream(stream)),
           "agile_module_launch")


def agile_selftest_bounded_waits(d_log, d_flag, flag_us: int, d_result, stream=None) -> None:
    _check(lib().agile_selftest_bounded_waits(_dptr(d_log), _dptr(d_flag), flag_us,
                                              _dptr(d_result), _stream(stream)),
           "agile_selftest_bounded_waits")
