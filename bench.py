"""Benchmark of the kernel memory guard on B300.

Workload (one step): the guarded streaming kernels -- copy a = b, scale a = s*b and
triad a = b + s*c -- over three fp32 arrays of 2^28 elements (1 GiB each) that live in
an arena described by a 1096-range guard table (1024 user allocations, 64 protected
ranges, 8 MMIO ranges; 2 MiB pages), poison policy, violation log reset each step.
Metric: guarded HBM GB/s = algorithmic bytes (8 + 8 + 12 bytes per element) / time.
Beside it: the unguarded twins (guarded/unguarded ratio), the batch check's
checks/s on the 1M-access table workload and on a 2^28-access stream, the roofline of
the dominant kernel, an end-to-end figure through host buffers, and the oracle timed on
the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import agile_synth as syn  # noqa: E402

N_ELEMS = 1 << 28
BYTES_PER_ELEM = {"copy": 8, "scale": 8, "triad": 12}
STEP_BYTES = sum(BYTES_PER_ELEM.values()) * N_ELEMS
PTX_STREAM = os.path.join(ROOT, "paper_2606_06697_b300", "ptx", "stream.ptx")
PTX_IRREGULAR = os.path.join(ROOT, "paper_2606_06697_b300", "ptx", "irregular.ptx")
METRIC = "guarded HBM GB/s (guarded streaming copy+scale+triad; guarded/unguarded ratio, " \
         "guard checks/s beside)"
WORKLOAD = ("guarded streaming copy/scale/triad, 3 fp32 arrays of 2^28 elements (1 GiB each) "
            "in an arena under a 1096-range guard table (1024 user, 64 protected, 8 MMIO), "
            "2 MiB pages, poison policy")
KERNEL_SOURCES = ["paper_2606_06697_b300/csrc/stream.cu",
                  "paper_2606_06697_b300/csrc/stream_body.cuh",
                  "paper_2606_06697_b300/csrc/guard_device.cuh"]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def source_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel_tag):
    """dram bytes per launch recorded by an ncu capture of the same kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = source_hash(KERNEL_SOURCES)
    for line in open(path):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == kernel_tag and f[1] == want:
            return int(f[2])
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.15)
        self.proc.terminate()
        self.proc.wait()
        self.file.seek(0)
        rows = [r.split(", ") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(name)
            except (IndexError, ValueError):
                continue
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x, device):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- oracle timing


def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _chunks(n: int, parts: int, align: int = 4):
    """Contiguous [lo, hi) pieces of range(n), boundaries multiples of `align`."""
    cuts = [min(n, (n * k // parts) // align * align) for k in range(parts)] + [n]
    return [(lo, hi) for lo, hi in zip(cuts, cuts[1:]) if hi > lo]


def _parallel(fn, pieces, workers):
    """fn over the pieces on `workers` threads. The oracle's C entry points release the
    interpreter lock while they run, so the pieces run on separate cores."""
    if workers <= 1:
        return [fn(p) for p in pieces]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(workers) as ex:
        return list(ex.map(fn, pieces))


class StreamSample:
    """The first n elements of the workload's b and c arrays, in the workload's arena
    layout (a 1096-range table), for the oracle's guarded copy / scale / triad."""

    def __init__(self, n: int, seed: int = 1):
        r, span, off = syn.stream_layout(N_ELEMS)
        self.base = 0x7F0000000000
        self.table = r.shifted(self.base)
        self.off = off
        st = syn.Stream(seed, 8)
        self.b = st.uniform(n).astype(np.float32)
        self.c = st.uniform(n).astype(np.float32)
        self.a0 = np.zeros(n, np.float32)
        self.n = n

    def run(self, workers: int):
        """One step (copy, scale, triad) of the oracle over the sample, the elements cut
        into one contiguous piece per thread. Returns (seconds, algorithmic bytes)."""
        import oracle

        def piece(op):
            def f(p):
                lo, hi = p
                va = {k: self.base + self.off[k] + 4 * lo for k in "abc"}
                return oracle.stream(op, self.table, va, self.b[lo:hi], self.c[lo:hi],
                                     self.a0[lo:hi], 3.0, "poison")
            return f
        pieces = _chunks(self.n, workers)
        t0 = time.perf_counter()
        for op in ("copy", "scale", "triad"):
            _parallel(piece(op), pieces, workers)
        return time.perf_counter() - t0, sum(BYTES_PER_ELEM.values()) * self.n


def cpu_batch_check(workers: int):
    """The oracle's batch check on the 84-range table workload (10 B per check): the
    sorted-interval form on every host thread over 2^24 accesses (the 1M generated
    accesses repeated), and single-threaded on the 1M accesses themselves, both the
    sorted form and the linear scan that defines the rule."""
    import oracle
    t = syn.batch_table()
    addr, width, _ = syn.batch_accesses(t, 1 << 20)
    out = {}
    for name, method, reps, w in (("linear_1_thread", "linear", 1, 1),
                                  ("sorted_1_thread", "sorted", 1, 1),
                                  ("sorted_all_threads", "sorted", 16, workers)):
        A, W = np.tile(addr, reps), np.tile(width, reps)
        pieces = _chunks(len(A), w, 1)
        t0 = time.perf_counter()
        _parallel(lambda p: oracle.check_batch(t, A[p[0]:p[1]], W[p[0]:p[1]], method=method),
                  pieces, w)
        dt = time.perf_counter() - t0
        out[name] = {"checks_per_s": len(A) / dt, "accesses": len(A), "threads": w,
                     "seconds": dt}
    return out


def run_reference(args, ws, rank):
    """The oracle as the reference arm, on every host thread: each step a bounded sample
    of the workload."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    workers = host_threads()
    dt, nb = StreamSample(1 << 20).run(workers)           # calibrate
    per_elem = dt / (1 << 20)
    budget = 90.0 / max(args.steps + args.warmup, 1)     # whole run ~1.5 min
    n_sample = int(max(1 << 16, min(1 << 26, budget / per_elem)))
    n_sample -= n_sample % 4
    sample = StreamSample(n_sample)
    for _ in range(args.warmup):
        sample.run(workers)
    tot_t, tot_b = 0.0, 0
    for _ in range(args.steps):
        dt, nb = sample.run(workers)
        tot_t += dt
        tot_b += nb
    value = tot_b / tot_t / 1e9
    desc = (f"first {n_sample} elements of each array per step (of 2^28), same arena table; "
            f"the oracle (sorted-interval search per 16-byte access) on {workers} host threads, "
            f"one contiguous piece each")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "elements": N_ELEMS, "sample_elements": n_sample},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": workers, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm


def run_ours(args, ws, rank, local):
    import torch

    import paper_2606_06697_b300 as ag

    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)        # torch's own work (fills, copies) goes on the same stream
    hbm_peak, peak_kind = peaks()

    r, span, off = syn.stream_layout(N_ELEMS)
    arena = torch.empty(span, dtype=torch.uint8, device=dev)
    base = arena.data_ptr()
    rt = r.shifted(base)
    tbl = ag.agile_guard_table_build(rt.base, rt.size, rt.kind, rt.ident, 21)
    tbuf = torch.empty(tbl.device_bytes(), dtype=torch.uint8, device=dev)
    dtab = tbl.upload(tbuf, stream)
    A, B, C = (arena[off[k]:off[k] + 4 * N_ELEMS].view(torch.float32) for k in "abc")
    g = torch.Generator(device=dev).manual_seed(1234 + rank)
    B.uniform_(-1, 1, generator=g)
    C.uniform_(-1, 1, generator=g)
    log = torch.empty(ag.LOG_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    ops = ("copy", "scale", "triad")

    def step(guarded, ev=None, shape=None):
        if guarded:
            ag.agile_violation_log_init(log, rank, stream)
        for op in ops:
            if ev is not None:
                ev[op][0].record(stream)
            if shape is None:
                ag.agile_stream_launch(op, dtab if guarded else None, A, B, C, N_ELEMS, 3.0,
                                       "poison", log if guarded else None, stream)
            else:
                ag.agile_stream_launch_shape(op, dtab if guarded else None, A, B, C, N_ELEMS, 3.0,
                                             "poison", log if guarded else None, *shape, stream)
            if ev is not None:
                ev[op][1].record(stream)

    def timed(guarded, steps, warmup, per_kernel=False, shape=None):
        for _ in range(warmup):
            step(guarded, shape=shape)
        evs = []
        barrier(ws)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            ev = None
            if per_kernel:
                ev = {op: (torch.cuda.Event(enable_timing=True),
                           torch.cuda.Event(enable_timing=True)) for op in ops}
                evs.append(ev)
            step(guarded, ev, shape)
        t1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        ms = t0.elapsed_time(t1)
        kern = {op: statistics.mean(e[op][0].elapsed_time(e[op][1]) for e in evs) for op in ops} \
            if per_kernel else None
        return ms, kern

    # guarded: the headline, with clocks sampled during it
    clocks = Clocks(local)
    timed(True, 3, args.warmup)
    clocks.start()
    ms, kern = timed(True, args.steps, 0, per_kernel=True)
    ck = clocks.stop()
    ms = max_over_ranks(ws, ms, dev)
    rc, rec = ag.agile_violation_log_read(log, stream)
    assert rc == 0 and rec.count == 0, "unexpected violation in the guarded workload"
    value = ws * STEP_BYTES * args.steps / (ms / 1e3) / 1e9
    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "GB/s", "quick": True,
                              "elements": N_ELEMS, "steps": args.steps, "kernel_ms": kern,
                              "clocks": ck}), flush=True)
        return

    # unguarded twins at both launch shapes (4 units x 2 blocks/SM is their own best shape,
    # 8 x 1 is the guarded kernels'), and the guarded kernels at the unguarded shape
    shapes = {"u8_b1": (8, 1), "u4_b2": (4, 2)}
    by_shape = {}
    kern_u, value_u = {op: None for op in ops}, None
    if "unguarded" in args.legs:
        k_u = max(args.steps // 2, 10)
        for name, sh in shapes.items():
            ms_s, kern_s = timed(False, k_u, 3, per_kernel=True, shape=sh)
            by_shape[f"unguarded_{name}"] = {"gbs": STEP_BYTES * k_u / (ms_s / 1e3) / 1e9,
                                             "kernel_ms": kern_s}
        ms_s, kern_s = timed(True, k_u, 3, per_kernel=True, shape=shapes["u4_b2"])
        by_shape["guarded_u4_b2"] = {"gbs": STEP_BYTES * k_u / (ms_s / 1e3) / 1e9, "kernel_ms": kern_s}
        by_shape["guarded_u8_b1"] = {"gbs": value / ws, "kernel_ms": kern}
        best = max(("u8_b1", "u4_b2"), key=lambda k: by_shape[f"unguarded_{k}"]["gbs"])
        value_u = by_shape[f"unguarded_{best}"]["gbs"]
        kern_u = by_shape[f"unguarded_{best}"]["kernel_ms"]

    # the same kernels from hand-written PTX through the guard pass (poison)
    ptx_kern, ptx_gbs, ptx_plain_gbs, ptx_ap_gbs = None, None, None, None
    if "ptx" in args.legs:
        ptx_kern = ptx_injected(ag, torch, dev, stream, dtab, log, A, B, C)
        ptx_gbs = STEP_BYTES / (sum(v for k, v in ptx_kern.items() if k.endswith("guarded")) / 1e3) / 1e9
        ptx_ap_gbs = STEP_BYTES / (sum(v for k, v in ptx_kern.items() if k.endswith("aperture")) / 1e3) / 1e9
        ptx_plain_gbs = STEP_BYTES / (sum(v for k, v in ptx_kern.items() if k.endswith("plain")) / 1e3) / 1e9

    # dominant kernel roofline
    top = max(kern, key=kern.get)
    achieved = BYTES_PER_ELEM[top] * N_ELEMS / (kern[top] / 1e3) / 1e9
    traffic = traffic_from_profile(f"stream_{top}_guarded")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "kernel": f"k_stream<{top}, guarded>",
                "peak_kind": f"{peak_kind} hbm_gbs (copy, burst)"}

    # batch check throughput: the 1M-access table workload and a 2^28-access stream
    batch = batch_throughput(ag, torch, dev, stream) if "batch" in args.legs else None
    irregular = irregular_sweep(ag, torch, dev, stream, n=args.irregular_n,
                                stripes=args.irregular_stripes, kinds=args.irregular_kinds.split(","),
                                dists=args.irregular_dists.split(","),
                                stress="gather" in args.irregular_kinds and args.irregular_stress) \
        if "irregular" in args.legs else None
    clients = batch_clients(ag, torch, dev, stream) if "clients" in args.legs else None
    serving = serve_sweep(ag, torch, dev) if "serving" in args.legs else None

    # end to end through host buffers: H2D of b, c, the three guarded kernels, D2H of a
    e2e = end_to_end(ag, torch, ws, dev, stream, dtab, log, A, B, C, max(3, min(args.steps // 100, 10))) \
        if "e2e" in args.legs else None

    cpu = None
    if rank == 0 and "cpu" in args.legs:
        import oracle
        oracle.build()
        workers = host_threads()
        n_all, n_one = 1 << 27, 1 << 25
        dt, nb = StreamSample(n_all).run(workers)
        dt1, nb1 = StreamSample(n_one).run(1)
        cpu = {"value": nb / dt / 1e9, "unit": "GB/s", "cores": workers, "kind": "oracle",
               "sample": f"guarded copy+scale+triad over the first 2^27 of the 2^28 elements, "
                         f"same arena table; the oracle on {workers} host threads (one "
                         f"contiguous piece each), {dt:.1f} s",
               "single_thread": {"value": nb1 / dt1 / 1e9, "unit": "GB/s", "cores": 1,
                                 "sample": f"first 2^25 elements, {dt1:.1f} s"},
               "batch_check": cpu_batch_check(workers)}

    if rank == 0:
        hb = hbm_peak
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "elements": N_ELEMS, "table_ranges": len(r),
                       "page_bytes": 1 << 21, "policy": "poison",
                       "l2": "each array 1 GiB, larger than the 126 MB L2; no flush needed"},
            # the full measurements first; the figures the targets are read from last
            "serving": serving, "irregular": irregular, "batch_clients": clients,
            "batch_check": batch, "ptx_kernel_ms": ptx_kern, "stream_shapes": by_shape,
            "kernel_ms": {f"{op}_guarded": kern[op] for op in ops} |
                         {f"{op}_unguarded": kern_u[op] for op in ops},
            "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
            "gpu_launches": args.steps * 4, "clocks": ck,
            "targets": targets_summary(value / ws, value_u, by_shape, ptx_gbs, ptx_plain_gbs,
                                       ptx_ap_gbs, batch, irregular, clients, serving, cpu, hb),
        }
        print(json.dumps(line), flush=True)


def _r(x, d=3):
    return None if x is None else round(float(x), d)


def targets_summary(guarded, unguarded_best, by_shape, ptx_gbs, ptx_plain_gbs, ptx_ap_gbs,
                    batch, irregular, clients, serving, cpu, hbm_peak):
    """The ratios and rates the targets are judged on, compactly."""
    t = {"guarded_gbs": _r(guarded, 1), "guarded_frac_of_peak": _r(guarded / hbm_peak),
         "unguarded_best_gbs": _r(unguarded_best, 1),
         "guarded_over_unguarded_best": _r(guarded / unguarded_best) if unguarded_best else None,
         "unguarded_gbs_by_shape": {k[len("unguarded_"):]: _r(v["gbs"], 1)
                                    for k, v in by_shape.items() if k.startswith("unguarded_")},
         "ptx_table_over_plain": _r(ptx_gbs / ptx_plain_gbs) if ptx_gbs else None,
         "ptx_aperture_over_plain": _r(ptx_ap_gbs / ptx_plain_gbs) if ptx_ap_gbs else None}
    if batch:
        t["batch_gchecks"] = {
            size: {"table": _r(row[row["best"]]["checks_per_s"] / 1e9, 1),
                   "table_frac_of_peak": _r(row[row["best"]]["gbs"] / hbm_peak),
                   "aperture": _r(row["aperture_rule"]["checks_per_s"] / 1e9, 1)}
            for size, row in batch.items()}
    if irregular:
        t["irregular_guarded_over_unguarded"] = {
            k: _r(v["guarded_over_unguarded"]) for k, v in irregular.items()}
        t["irregular_ptx_table_over_plain"] = {
            k: _r(v["ptx_table_over_plain"]) for k, v in irregular.items() if "ptx_table_over_plain" in v}
        t["irregular_ptx_table_over_plain_2_blocks_per_sm"] = {
            k: _r(v["ptx_table_over_plain_two_blocks_per_sm"]) for k, v in irregular.items()
            if "ptx_table_over_plain_two_blocks_per_sm" in v}
    if clients:
        t["clients_graph_speedup"] = _r(clients["speedup_graph_vs_separate"], 2)
    if serving:
        t["serving_p99_us"] = {k: [_r(v["continuous"]["p99_us"], 0), _r(v["one_at_a_time"]["p99_us"], 0)]
                               for k, v in serving.items() if isinstance(v, dict) and "continuous" in v}
    if cpu:
        t["cpu_oracle"] = {"all_threads_gbs": _r(cpu["value"]), "threads": cpu["cores"],
                           "one_thread_gbs": _r(cpu["single_thread"]["value"]),
                           "batch_mchecks_all_threads": _r(cpu["batch_check"]["sorted_all_threads"]["checks_per_s"] / 1e6, 1),
                           "batch_mchecks_linear_1_thread": _r(cpu["batch_check"]["linear_1_thread"]["checks_per_s"] / 1e6, 1)}
    return t


def end_to_end(ag, torch, ws, dev, stream, dtab, log, A, B, C, steps):
    """The workload through the public API from pinned host buffers, every step:
    agile_stream_launch_host runs copy with b from the host, scale on the device-resident
    b, and triad with c from the host and a back to the host. Each call cuts its arrays
    into chunks whose copies in, guarded kernels and copies out overlap on three streams."""
    hb = torch.empty(N_ELEMS, dtype=torch.float32, pin_memory=True)
    hc = torch.empty(N_ELEMS, dtype=torch.float32, pin_memory=True)
    ha = torch.empty(N_ELEMS, dtype=torch.float32, pin_memory=True)
    hb.copy_(B.cpu())
    hc.copy_(C.cpu())

    def one():
        ag.agile_violation_log_init(log, 0, stream)
        ag.agile_stream_launch_host("copy", dtab, A, B, C, None, hb, None, N_ELEMS, 3.0,
                                    "poison", log, 0, stream)
        ag.agile_stream_launch_host("scale", dtab, A, B, C, None, None, None, N_ELEMS, 3.0,
                                    "poison", log, 0, stream)
        ag.agile_stream_launch_host("triad", dtab, A, B, C, ha, None, hc, N_ELEMS, 3.0,
                                    "poison", log, 0, stream)

    one()
    torch.cuda.synchronize()
    barrier(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ws, e0.elapsed_time(e1), dev)
    rc, rec = ag.agile_violation_log_read(log, stream)
    assert rc == 0 and rec.count == 0, "violation in the end-to-end run"
    return {"value": ws * STEP_BYTES * steps / (ms / 1e3) / 1e9, "unit": "GB/s",
            "h2d_bytes_per_step": 2 * 4 * N_ELEMS, "d2h_bytes_per_step": 4 * N_ELEMS,
            "steps": steps, "api": "agile_stream_launch_host (chunks of 2^24 elements, 3 streams)"}


def ptx_injected(ag, torch, dev, stream, dtab, log, A, B, C, reps=20):
    """Mean kernel time of the hand-written PTX copy/scale/triad, instrumented by the guard
    pass (poison) and as written (no guard), CUDA events."""
    import ctypes
    src = open(PTX_STREAM).read()
    guarded = ag.agile_module_load(ag.agile_guard_instrument_ptx(src, "poison")[0])
    ap = syn.table1_protected()
    aperture = ag.agile_module_load(ag.agile_guard_instrument_ptx(
        src, "poison", apertures=(ap.base, ap.size, ap.kind, ap.ident))[0])
    plain = ag.agile_module_load(src)
    ag.agile_violation_log_init(log, 0, stream)
    ag.agile_module_bind(guarded, dtab, log, stream)
    ag.agile_module_bind(aperture, None, log, stream)
    grid = torch.cuda.get_device_properties(dev).multi_processor_count * 4
    args = [ctypes.c_uint64(A.data_ptr()), ctypes.c_uint64(B.data_ptr()),
            ctypes.c_uint64(C.data_ptr()), ctypes.c_uint64(N_ELEMS), ctypes.c_float(3.0)]
    out = {}
    for name, mod in (("guarded", guarded), ("aperture", aperture), ("plain", plain)):
        for op in ("copy", "scale", "triad"):
            for _ in range(3):
                ag.agile_module_launch(mod, f"agile_ptx_{op}", grid, 512, args, stream)
            evs = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ag.agile_module_launch(mod, f"agile_ptx_{op}", grid, 512, args, stream)
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            out[f"{op}_{name}"] = statistics.mean(a.elapsed_time(b) for a, b in evs)
    rc, rec = ag.agile_violation_log_read(log, stream)
    assert rc == 0 and rec.count == 0, "violation in the PTX-injected run"
    guarded.unload()
    aperture.unload()
    plain.unload()
    return out


def batch_clients(ag, torch, dev, stream, n_clients=256, reps=5):
    """256 clients (50% copy, 30% gather, 20% histogram; lognormal buffers, median 2 MiB;
    tables of 8-4096 ranges): one persistent guarded launch (autotuned, then replayed as a
    CUDA graph) against 256 separate guarded launches."""
    from paper_2606_06697_b300.clients import ClientSet
    specs = syn.client_specs(n_clients)
    cs = ClientSet(specs, dev, log2_pages=(16, 21))
    n = len(cs.clients)
    buf = torch.empty(ag.agile_batch_device_bytes(n), dtype=torch.uint8, device=dev)
    best = ag.agile_batch_autotune([cs.work(0), cs.work(1)], [4096, 16384, 65536, 262144], buf,
                                   reps=3, stream=stream)
    v = best["variant"]
    ag.agile_batch_upload(cs.work(v), best["tile"], buf, stream)
    nbytes = cs.algorithmic_bytes()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        out = []
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    def separate():
        for i in range(n):
            cs.run_single(i, v, stream=stream)

    def batched():
        ag.agile_batch_launch(buf, n, best["tile"], best["span_checks"], best["blocks_per_sm"], stream)

    g = ag.agile_batch_graph_create(buf, n, best["tile"], best["span_checks"], best["blocks_per_sm"])
    ms_sep = timed(separate)
    ms_bat = timed(batched)
    ms_graph = timed(lambda: g.launch(stream))
    g.destroy()
    return {"clients": n, "algorithmic_bytes": nbytes, "tuned": best,
            "separate_launches_ms": ms_sep, "batched_ms": ms_bat, "graph_replay_ms": ms_graph,
            "separate_gbs": nbytes / ms_sep / 1e6, "graph_gbs": nbytes / ms_graph / 1e6,
            "speedup_graph_vs_separate": ms_sep / ms_graph,
            "mix": {o: sum(1 for s_ in specs if s_["op"] == o) for o in ("copy", "gather", "hist")}}



def irregular_sweep(ag, torch, dev, stream, n=1 << 28, reps=5, stripes=4096,
                    kinds=("gather", "scatter", "hist"), dists=("uniform", "zipf"), stress=True):
    """Gather / scatter / histogram over the 16 GiB striped table (4096 user allocations of
    4 MiB, each followed by a 64 KiB protected range), 2^28 int64 indices, uniform and
    Zipf(1.1), 0.1% aimed into protected ranges; guarded (poison, 2 MiB and 64 KiB pages)
    against unguarded. Indices are drawn on the device with a seeded torch generator."""
    r, span, off = syn.irregular_layout(n, stripes)
    ue = (4 << 20) // 4
    se, pe, bins = ((4 << 20) + (64 << 10)) // 4, (64 << 10) // 4, 1 << 20
    arena = torch.empty(span, dtype=torch.uint8, device=dev)
    base = arena.data_ptr()
    g = torch.Generator(device=dev).manual_seed(syn.SEED_BASE + 3)
    arena[:off["bins"]].view(torch.float32).uniform_(1, 2, generator=g)
    idx = arena[off["idx"]:off["idx"] + 8 * n].view(torch.int64)
    out_t = arena[off["out"]:off["out"] + 4 * n].view(torch.float32)
    bins_t = arena[off["bins"]:off["bins"] + 4 * bins].view(torch.int32)
    rr = r.shifted(base)
    tabs = {}
    for lg in (21, 16):
        t = ag.agile_guard_table_build(rr.base, rr.size, rr.kind, rr.ident, lg)
        b = torch.empty(t.device_bytes(), dtype=torch.uint8, device=dev)
        tabs[lg] = (t, b, t.upload(b, stream))
    log = torch.empty(ag.LOG_BYTES, dtype=torch.uint8, device=dev)
    useful = {"gather": 16, "scatter": 12, "hist": 8}
    res = {}
    # the hand-written PTX kernels: instrumented with the table guard, with the aperture
    # guard (the 4096 protected tails do not fit in four apertures, so the apertures are
    # the first four of them: a cheaper check, not the same protection), and as written
    import ctypes
    src = open(PTX_IRREGULAR).read()
    keep = np.flatnonzero(rr.kind != 0)[:4]
    apset = (rr.base[keep], rr.size[keep], rr.kind[keep], rr.ident[keep])
    ptx_mods = {"ptx_table_64KiB": ag.agile_module_load(ag.agile_guard_instrument_ptx(src, "poison")[0]),
                "ptx_aperture4": ag.agile_module_load(ag.agile_guard_instrument_ptx(
                    src, "poison", apertures=apset)[0]),
                "ptx_plain": ag.agile_module_load(src)}
    grid = torch.cuda.get_device_properties(dev).multi_processor_count * 4
    for dist in dists:
        if dist == "uniform":
            rank = torch.randint(0, stripes * ue, (n,), generator=g, device=dev, dtype=torch.int64)
        else:
            k = syn.zipf_torch(g, 1.1, stripes * ue, n, dev) - 1
            rank = (k * syn.ODD_MIX) & (stripes * ue - 1)
        element = (rank // ue) * se + rank % ue
        key = rank & (bins - 1)
        bad = torch.unique(torch.randint(0, n, (n // 1000,), generator=g, device=dev))
        nb = bad.numel()
        element[bad] = torch.randint(0, stripes, (nb,), generator=g, device=dev) * se + ue + \
            torch.randint(0, pe, (nb,), generator=g, device=dev)
        key[bad] = bins + torch.randint(0, pe, (nb,), generator=g, device=dev)
        del rank
        for kind in kinds:
            idx.copy_(key if kind == "hist" else element)
            target = base + (off["bins"] if kind == "hist" else 0)
            row = {}
            for label, lg in (("unguarded", None), ("guarded_2MiB", 21), ("guarded_64KiB", 16)):
                dtab = tabs[lg][2] if lg else None

                def once():
                    if lg:
                        ag.agile_violation_log_init(log, 0, stream)
                    ag.agile_irregular_launch(kind, dtab, idx, target, out_t, n, "poison",
                                              log if lg else None, stream)
                if kind == "hist":
                    bins_t.zero_()
                once()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                ts = []
                for _ in range(reps):
                    e0.record(stream)
                    once()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = statistics.median(ts)
                cell = {"ms": ms, "useful_gbs": useful[kind] * n / ms / 1e6}
                if lg:
                    rc, rec = ag.agile_violation_log_read(log, stream)
                    assert rec.count == nb, (kind, dist, rec.count, nb)
                    cell["violations"] = rec.count
                row[label] = cell
            row["guarded_over_unguarded"] = row["unguarded"]["ms"] / min(
                row["guarded_2MiB"]["ms"], row["guarded_64KiB"]["ms"])
            # the same guarded kernel with the __match_any_sync bitmap read (64 KiB pages)
            def once_match():
                ag.agile_violation_log_init(log, 0, stream)
                ag.agile_irregular_launch_fastpath(kind, tabs[16][2], idx, target, out_t, n, "poison",
                                                   log, "match", stream)
            if kind == "hist":
                bins_t.zero_()
            once_match()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                once_match()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            rc, rec = ag.agile_violation_log_read(log, stream)
            assert rec.count == nb, ("match", kind, dist, rec.count, nb)
            ms = statistics.median(ts)
            row["guarded_64KiB_match"] = {"ms": ms, "useful_gbs": useful[kind] * n / ms / 1e6}
            row["match_over_bitmap"] = row["guarded_64KiB"]["ms"] / ms
            args_ = [ctypes.c_uint64(idx.data_ptr()), ctypes.c_uint64(target),
                     ctypes.c_uint64(out_t.data_ptr()), ctypes.c_uint64(n)]
            for label, mod in ptx_mods.items():
                if label != "ptx_plain":
                    ag.agile_module_bind(mod, tabs[16][2] if label == "ptx_table_64KiB" else None, log)
                    ag.agile_violation_log_init(log, 0, stream)

                def once_ptx():
                    ag.agile_module_launch(mod, f"agile_ptx_{kind}", grid, 512, args_, stream)
                if kind == "hist":
                    bins_t.zero_()
                once_ptx()
                torch.cuda.synchronize()
                ts = []
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    once_ptx()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = statistics.median(ts)
                row[label] = {"ms": ms, "useful_gbs": useful[kind] * n / ms / 1e6}
                if label == "ptx_table_64KiB":      # every launch logged every denial
                    rc, rec = ag.agile_violation_log_read(log, stream)
                    assert rec.count == nb * (reps + 1), ("ptx", kind, dist, rec.count, nb)
                    row[label]["violations_per_launch"] = rec.count // (reps + 1)
            row["ptx_table_over_plain"] = row["ptx_plain"]["ms"] / row["ptx_table_64KiB"]["ms"]
            # the same two modules launched with half the blocks (two 512-thread blocks per
            # SM): as many as the instrumented kernel keeps resident at its register count
            half = {}
            for label in ("ptx_table_64KiB", "ptx_plain"):
                mod = ptx_mods[label]
                if label != "ptx_plain":
                    ag.agile_module_bind(mod, tabs[16][2], log)
                if kind == "hist":
                    bins_t.zero_()
                ag.agile_module_launch(mod, f"agile_ptx_{kind}", grid // 2, 512, args_, stream)
                torch.cuda.synchronize()
                ts = []
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ag.agile_module_launch(mod, f"agile_ptx_{kind}", grid // 2, 512, args_, stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                half[label] = statistics.median(ts)
            row["ptx_two_blocks_per_sm_ms"] = half
            row["ptx_table_over_plain_two_blocks_per_sm"] = half["ptx_plain"] / half["ptx_table_64KiB"]
            res[f"{kind}_{dist}"] = row
        del element, key
    for mod in ptx_mods.values():
        mod.unload()
    del arena, idx, out_t, bins_t
    torch.cuda.empty_cache()
    if stress:
        res["gather_uniform_stress_60k_4k"] = irregular_stress(ag, torch, dev, stream, n, reps)
        torch.cuda.empty_cache()
    return res


def irregular_stress(ag, torch, dev, stream, n, reps, stripes=1 << 18):
    """The adversarial variant of the irregular table: 2^18 stripes of a 60 KiB user range
    and a 4 KiB protected range (16 GiB, 524288 ranges), uniform gather of 2^28 indices,
    0.1% into the protected ranges. With 64 KiB pages (and bitmap blocks) no page is all
    user; 4 KiB pages make every page pure again."""
    user, prot = 60 << 10, 4 << 10
    r, span, off = syn.irregular_layout(n, stripes, user, prot, 1 << 10)
    arena = torch.empty(span, dtype=torch.uint8, device=dev)
    base = arena.data_ptr()
    g = torch.Generator(device=dev).manual_seed(syn.SEED_BASE + 13)
    arena[:off["bins"]].view(torch.float32).uniform_(1, 2, generator=g)
    ue, se, pe = user // 4, (user + prot) // 4, prot // 4
    rank = torch.randint(0, stripes * ue, (n,), generator=g, device=dev, dtype=torch.int64)
    idx = arena[off["idx"]:off["idx"] + 8 * n].view(torch.int64)
    idx.copy_((rank // ue) * se + rank % ue)
    del rank
    bad = torch.unique(torch.randint(0, n, (n // 1000,), generator=g, device=dev))
    idx[bad] = torch.randint(0, stripes, (bad.numel(),), generator=g, device=dev) * se + ue + \
        torch.randint(0, pe, (bad.numel(),), generator=g, device=dev)
    out_t = arena[off["out"]:off["out"] + 4 * n].view(torch.float32)
    rr = r.shifted(base)
    log = torch.empty(ag.LOG_BYTES, dtype=torch.uint8, device=dev)
    row = {"ranges": int(len(rr.base))}
    for label, lg in (("unguarded", None), ("guarded_auto", 0), ("guarded_4KiB", 12),
                      ("guarded_64KiB", 16)):
        dtab = None
        if lg is not None:
            t = ag.agile_guard_table_build(rr.base, rr.size, rr.kind, rr.ident, lg)
            if lg == 0:
                row["auto_log2_page"] = t.geometry()[0]
            tb = torch.empty(t.device_bytes(), dtype=torch.uint8, device=dev)
            dtab = t.upload(tb, stream)

        def once():
            if lg is not None:
                ag.agile_violation_log_init(log, 0, stream)
            ag.agile_irregular_launch("gather", dtab, idx, base, out_t, n, "poison",
                                      log if lg is not None else None, stream)
        once()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            once()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        cell = {"ms": ms, "useful_gbs": 16 * n / ms / 1e6}
        if lg is not None:
            rc, rec = ag.agile_violation_log_read(log, stream)
            assert rec.count == bad.numel(), (label, rec.count, bad.numel())
            cell["violations"] = rec.count
        row[label] = cell
    row["guarded_over_unguarded"] = row["unguarded"]["ms"] / row["guarded_auto"]["ms"]
    del arena
    torch.cuda.empty_cache()
    return row


def serve_sweep(ag, torch, dev, rates=(1e3, 3e3, 1e4, 3e4, 1e5), window_s=0.3, min_requests=6000):
    """64 clients' validate + guarded-launch requests with Poisson arrivals; 0.5% carry a
    bad pointer. Continuous batching against one request at a time, per arrival rate:
    p50/p99 arrival-to-completion latency, its breakdown, and throughput; at the top rate
    the served bytes per second against the HBM peak and the worker's time per request."""
    from paper_2606_06697_b300.serving import ServedClients, latency_stats, serve
    cs = ServedClients(syn.serve_specs(64), dev)
    out = {}
    for rate in rates:
        n = int(min(max(rate * window_s, min_requests), 30000))
        gen = syn.serve_requests(cs.layouts, rate, n)
        bad = sum(g["bad"] is not None for g in gen)
        row = {"requests": n, "bad_pointer_requests": bad}
        for mode, cont in (("continuous", True), ("one_at_a_time", False)):
            cs.reset()
            done, peak = serve(cs, gen, continuous=cont)
            st = latency_stats(gen, done, cs)
            assert st["rejected"] == bad, "a bad pointer was not rejected"
            row[mode] = st
        out[f"{int(rate)}_per_s"] = row
    return out


def batch_throughput(ag, torch, dev, stream, sizes=(1 << 20, 1 << 28), reps=None,
                     log2_pages=(12, 16, 21)):
    """Batch check (10 B/check: 8 address + 1 width in, 1 verdict out) on the 84-range
    table workload, at each page size; inputs replicated from 1M generated accesses, L2
    flushed before every launch. Returns per size and page size, plus the best page size,
    and beside them the aperture-only rule (Table I's two protected apertures) on the
    aperture workload of the same size."""
    t = syn.batch_table()
    log = torch.empty(ag.LOG_BYTES, dtype=torch.uint8, device=dev)
    tabs = {}
    for lg in log2_pages:
        tbl = ag.agile_guard_table_build(t.base, t.size, t.kind, t.ident, lg)
        buf = torch.empty(tbl.device_bytes(), dtype=torch.uint8, device=dev)
        tabs[lg] = (tbl, buf, tbl.upload(buf, stream))
    out = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for n in sizes:
        name = f"2^{n.bit_length() - 1}" if n & (n - 1) == 0 else str(n)
        m = min(n, 1 << 20)
        addr, width, _ = syn.batch_accesses(t, m)
        da = torch.from_numpy(addr.view(np.int64)).to(dev).repeat((n + m - 1) // m)[:n]
        dw = torch.from_numpy(width).to(dev).repeat((n + m - 1) // m)[:n]
        dv = torch.empty(n, dtype=torch.uint8, device=dev)
        nrep = reps or (20 if n <= 1 << 20 else 5)
        res = {}
        for lg, (_, _, dtab) in tabs.items():
            tot = 0.0
            for i in range(nrep + 3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    flush.fill_(i & 0xFF)                      # evict the inputs from L2, on
                    ag.agile_violation_log_init(log, 0, stream)  # the check's own stream
                    e0.record(stream)
                    ag.agile_guard_check_batch(dtab, da, dw, n, dv, log, stream)
                    e1.record(stream)
                torch.cuda.synchronize()
                if i >= 3:
                    tot += e0.elapsed_time(e1)
            ms = tot / nrep
            res[f"page_2^{lg}"] = {"checks_per_s": n / (ms / 1e3), "ms": ms,
                                   "gbs": n * 10 / (ms / 1e3) / 1e9}
        best = min(res, key=lambda k: res[k]["ms"])
        a_addr, a_width, _ = syn.aperture_accesses(m)
        da.copy_(torch.from_numpy(a_addr.view(np.int64)).to(dev).repeat((n + m - 1) // m)[:n])
        dw.copy_(torch.from_numpy(a_width).to(dev).repeat((n + m - 1) // m)[:n])
        apset = syn.table1_protected()
        tot = 0.0
        for i in range(nrep + 3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
                ag.agile_violation_log_init(log, 0, stream)
                e0.record(stream)
                ag.agile_aperture_check_batch((apset.base, apset.size, apset.kind, apset.ident),
                                              da, dw, n, dv, log, stream)
                e1.record(stream)
            torch.cuda.synchronize()
            if i >= 3:
                tot += e0.elapsed_time(e1)
        ms = tot / nrep
        aperture = {"checks_per_s": n / (ms / 1e3), "ms": ms, "gbs": n * 10 / (ms / 1e3) / 1e9}
        out[name] = dict(res, best=best, bytes_per_check=10, aperture_rule=aperture)
        del da, dw, dv
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=800)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--elements", type=int, default=1 << 28,
                    help="elements per array (the workload is 2^28; smaller only for profiling)")
    ap.add_argument("--quick", action="store_true",
                    help="guarded steps only: no unguarded, PTX, batch, e2e or CPU legs")
    ap.add_argument("--batch-only", type=int, default=0, metavar="N",
                    help="only time the batch check on N accesses (profiling)")
    ap.add_argument("--batch-page", type=int, default=16, help="log2 page size for --batch-only")
    ap.add_argument("--legs", default="all",
                    help="comma list of extra legs: unguarded,ptx,batch,irregular,clients,serving,"
                         "e2e,cpu (the guarded steps always run)")
    ap.add_argument("--irregular-n", type=int, default=1 << 28)
    ap.add_argument("--irregular-stripes", type=int, default=4096)
    ap.add_argument("--irregular-kinds", default="gather,scatter,hist")
    ap.add_argument("--irregular-dists", default="uniform,zipf")
    ap.add_argument("--irregular-stress", type=int, default=1,
                    help="0: leave out the 16 GiB stress layout (small profiling runs)")
    args = ap.parse_args()
    args.legs = {"unguarded", "ptx", "batch", "irregular", "clients", "serving", "e2e", "cpu"} \
        if args.legs == "all" else set(args.legs.split(","))
    global N_ELEMS, STEP_BYTES
    N_ELEMS = args.elements - args.elements % 4
    STEP_BYTES = sum(BYTES_PER_ELEM.values()) * N_ELEMS
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":                     # host-only: rank 0 runs, others exit
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")),
                      int(os.environ.get("RANK", "0")))
        return
    ws, rank, local = dist_setup()
    if args.batch_only:
        import torch
        import paper_2606_06697_b300 as ag
        torch.cuda.set_device(local)
        st = torch.cuda.Stream()
        torch.cuda.set_stream(st)
        print(json.dumps({"batch_check": batch_throughput(ag, torch, f"cuda:{local}", st,
                                                          sizes=(args.batch_only,), reps=args.steps,
                                                          log2_pages=(args.batch_page,))}))
        return
    run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
