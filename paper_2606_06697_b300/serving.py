"""Host-side set-up of served clients: each client's resident arena (inputs, output
slots, decoys), its host and device tables (freed allocations left out), its log, and
the conversion of generated requests into agile_request_t. Orchestration only: the
validation, admission, batching and guarded kernels run in the library's worker.
"""
from __future__ import annotations

import numpy as np
import torch

import agile_synth as syn

from . import abi

_ROUND = 2 << 20


class ServedClients:
    def __init__(self, specs, device="cuda:0", log2_page=21, seed=syn.SEED_BASE + 5):
        self.specs = specs
        self.device = device
        lay = [syn.serve_layout(s, seed) for s in specs]
        self.layouts = lay
        offs, cur = [], 0
        for lt in lay:
            offs.append(cur)
            cur += (lt[2] + _ROUND - 1) // _ROUND * _ROUND
        self.arena = torch.empty(cur, dtype=torch.uint8, device=device)
        self.base = self.arena.data_ptr()
        self.off = offs
        self.tables, self.devs = [], []
        sizes = []
        for (r, freed, span, boff, bsz, n), off in zip(lay, offs):
            live = ~freed
            rr = r.shifted(self.base + off)
            t = abi.agile_guard_table_build(rr.base[live], rr.size[live], rr.kind[live],
                                            rr.ident[live], log2_page)
            self.tables.append(t)
            sizes.append((t.device_bytes() + 255) // 256 * 256)
        self.table_buf = torch.empty(sum(sizes), dtype=torch.uint8, device=device)
        pos = 0
        for t, sz in zip(self.tables, sizes):
            self.devs.append(t.upload(self.table_buf.data_ptr() + pos))
            pos += sz
        self.logs = torch.empty(len(specs) * abi.LOG_BYTES, dtype=torch.uint8, device=device)
        g = torch.Generator(device=device).manual_seed(seed & 0xFFFF)
        for i, (s, (r, freed, span, boff, bsz, n)) in enumerate(zip(specs, lay)):
            if s["op"] == "copy":
                self.view(i, "b", torch.float32, n).uniform_(-1, 1, generator=g)
            elif s["op"] == "gather":
                self.view(i, "t", torch.float32, s["bytes"] // 4).uniform_(-1, 1, generator=g)
            if s["op"] in ("gather", "hist"):
                hi = s["bytes"] // 4 if s["op"] == "gather" else syn.HIST_BINS
                st = syn.Stream(seed, 500 + i)
                self.view(i, "idx", torch.int64, n).copy_(torch.from_numpy(st.below(hi, n)))
        self.reset()
        torch.cuda.synchronize(device)

    def addr(self, i, off):
        return self.base + self.off[i] + off

    def view(self, i, name, dtype, count):
        o = self.off[i] + self.layouts[i][3][name]
        nb = count * torch.tensor([], dtype=dtype).element_size()
        return self.arena[o:o + nb].view(dtype)

    def log(self, i):
        return self.logs[i * abi.LOG_BYTES:(i + 1) * abi.LOG_BYTES]

    def reset(self):
        self.logs.zero_()
        for i in range(len(self.specs)):
            abi.agile_violation_log_init(self.log(i), i)
            for k in range(syn.SERVE_SLOTS):
                o = self.off[i] + self.layouts[i][3][f"out{k}"]
                self.arena[o:o + self.layouts[i][4][f"out{k}"]].zero_()

    def work(self, i, slot, log=None):
        s = self.specs[i]
        _, _, _, boff, bsz, n = self.layouts[i]
        a = lambda k: self.addr(i, boff[k])
        if s["op"] == "copy":
            return abi.make_work("copy", self.devs[i], a(f"out{slot}"), a("b"), None, n, 3.0,
                                 "poison", log, i)
        if s["op"] == "gather":
            return abi.make_work("gather", self.devs[i], a(f"out{slot}"), a("idx"), a("t"), n, 0.0,
                                 "poison", log, i)
        return abi.make_work("hist", self.devs[i], None, a("idx"), a(f"out{slot}"), n, 0.0,
                             "poison", log, i)

    def request(self, tag, g):
        """agile_request_t from a generated request dict."""
        i, slot = g["client"], g["slot"]
        r = abi.Request()
        r.tag = tag
        r.client = i
        r.nargs = len(g["args"])
        for k, (off, nb) in enumerate(g["args"]):
            r.arg_ptr[k] = self.addr(i, off)
            r.arg_bytes[k] = nb
        r.work = self.work(i, slot)
        r.work.table = None                  # the worker fills in the client's table and log
        r.work.log = None
        _, _, _, boff, bsz, n = self.layouts[i]
        r.mem_bytes = sum(nb for k, nb in bsz.items() if not k.startswith("out")) + \
            bsz[f"out{slot}"]
        r.excl = (i << 8 | slot) + 1
        r.arrival_ns = g["arrival_ns"]
        return r

    def kernel_bytes(self, i):
        """Algorithmic bytes of client i's kernel: copy 8, gather 16, histogram 8 per element."""
        n = self.layouts[i][5]
        return n * {"copy": 8, "gather": 16, "hist": 8}[self.specs[i]["op"]]

    def output(self, i, slot):
        o = self.off[i] + self.layouts[i][3][f"out{slot}"]
        return self.arena[o:o + self.layouts[i][4][f"out{slot}"]]


def serve(clients: ServedClients, gen_reqs, continuous=True, max_batch=64, max_inflight=4,
          tile=16384, budget=160 * 10**9, timeout_s=120.0):
    """Run generated requests through a native worker; returns the completions."""
    import time
    cfg = abi.WorkerConfig(budget, max_batch, max_inflight, tile, int(continuous))
    d_buf = torch.empty(abi.agile_worker_device_bytes(cfg), dtype=torch.uint8, device=clients.device)
    w = abi.Worker(cfg, clients.tables, clients.devs, [clients.log(i) for i in range(len(clients.specs))],
                   d_buf)
    w.submit([clients.request(k, g) for k, g in enumerate(gen_reqs)])
    w.start()
    done = []
    t_end = time.time() + timeout_s
    while len(done) < len(gen_reqs) and time.time() < t_end:
        done += w.poll(4096, 50)
    peak = w.clock()[2]
    w.destroy()
    return done, peak


def latency_stats(gen_reqs, done, clients=None):
    """p50 / p99 arrival-to-completion latency of the served requests, throughput, the
    rejections, and where the time goes: pickup (arrival to validated by the worker),
    wait (validated to packed into a launch), launch (the copy and kernel queued) and run
    (queued to the request's completion notice), each as p50 / p99 in microseconds. With
    `clients`, the algorithmic bytes the served kernels moved per second."""
    ok = [c for c in done if c.status == 0]
    lat = np.array([(c.done_ns - c.arrival_ns) / 1e3 for c in ok])
    span = (max(c.done_ns for c in done) - min(g["arrival_ns"] for g in gen_reqs)) / 1e9
    rej = [c for c in done if c.status == 1]

    def pct(x):
        x = np.asarray(x, dtype=np.float64) / 1e3
        return [round(float(np.percentile(x, 50)), 1), round(float(np.percentile(x, 99)), 1)] \
            if len(x) else None
    out = {"requests": len(gen_reqs), "served": len(ok), "rejected": len(rej),
           "p50_us": float(np.percentile(lat, 50)) if len(lat) else None,
           "p99_us": float(np.percentile(lat, 99)) if len(lat) else None,
           "throughput_rps": len(done) / span if span > 0 else None,
           "launches": len({c.launch for c in ok}),
           "breakdown_p50_p99_us": {
               "pickup": pct([c.seen_ns - c.arrival_ns for c in ok]),
               "wait": pct([c.admit_ns - c.seen_ns for c in ok]),
               "launch": pct([c.queued_ns - c.admit_ns for c in ok]),
               "run": pct([c.done_ns - c.queued_ns for c in ok])}}
    out["requests_per_launch"] = len(ok) / out["launches"] if out["launches"] else None
    if clients is not None and span > 0:
        moved = sum(clients.kernel_bytes(gen_reqs[c.tag]["client"]) for c in ok)
        out["served_gbs"] = moved / span / 1e9
    return out
