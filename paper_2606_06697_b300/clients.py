"""Host-side set-up of many clients for the batched guarded launch: one device arena
carved into per-client arenas, one guard table per client (per page size), one log per
client, and the work items. Memory comes from PyTorch; every check and kernel runs in
the library. This is orchestration only -- it computes no verdicts.
"""
from __future__ import annotations

import numpy as np
import torch

import agile_synth as syn

from . import abi

_ROUND = 2 << 20


class ClientSet:
    """Clients from `agile_synth.client_specs`, resident on `device`.

    log2_pages: page sizes to build each client's table with (one work-list variant per
    page size). frac_bad: fraction of gather/histogram indices aimed at one of the
    client's protected decoy ranges (or a hole when it has none)."""

    def __init__(self, specs, device="cuda:0", log2_pages=(21,), frac_bad=0.0,
                 policy="poison", seed=syn.SEED_BASE + 4):
        self.specs = specs
        self.device = device
        self.policy = policy
        self.log2_pages = tuple(log2_pages)
        lay = [syn.client_layout(s, seed) for s in specs]
        offs, cur = [], 0
        for (_, span, _, _) in lay:
            offs.append(cur)
            cur += (span + _ROUND - 1) // _ROUND * _ROUND
        self.arena = torch.empty(cur, dtype=torch.uint8, device=device)
        base = self.arena.data_ptr()
        self.base = base
        self.clients = []
        tables = []
        for s, (r, span, boff, n), off in zip(specs, lay, offs):
            rr = r.shifted(base + off)
            c = {"spec": s, "ranges": rr, "arena_off": off, "span": span, "n": n,
                 "buf": {k: base + off + v for k, v in boff.items()}}
            ts = [abi.agile_guard_table_build(rr.base, rr.size, rr.kind, rr.ident, lg)
                  for lg in self.log2_pages]
            tables.append(ts)
            self.clients.append(c)
        sizes = [[(t.device_bytes() + 255) // 256 * 256 for t in ts] for ts in tables]
        self.table_buf = torch.empty(sum(map(sum, sizes)), dtype=torch.uint8, device=device)
        tb = self.table_buf.data_ptr()
        pos = 0
        for c, ts, sz in zip(self.clients, tables, sizes):
            c["dev"] = []
            for t, b in zip(ts, sz):
                c["dev"].append(t.upload(tb + pos))
                pos += b
            c["tables"] = ts
        self.logs = torch.empty(len(specs) * abi.LOG_BYTES, dtype=torch.uint8, device=device)
        self._fill(frac_bad, seed)
        torch.cuda.synchronize(device)

    # ------------------------------------------------------------------ data

    def view(self, c, name, dtype, count):
        off = c["buf"][name] - self.base
        nb = count * torch.tensor([], dtype=dtype).element_size()
        return self.arena[off:off + nb].view(dtype)

    def _fill(self, frac_bad, seed):
        g = torch.Generator(device=self.device).manual_seed(seed & 0xFFFF)
        for c in self.clients:
            s, n = c["spec"], c["n"]
            if s["op"] == "copy":
                self.view(c, "b", torch.float32, n).uniform_(-1, 1, generator=g)
            elif s["op"] == "gather":
                self.view(c, "t", torch.float32, s["bytes"] // 4).uniform_(-1, 1, generator=g)
            target_name = "t" if s["op"] == "gather" else "bins"
            if s["op"] in ("gather", "hist"):
                bad = None
                if frac_bad:
                    # a protected decoy of this client, else the hole after the target
                    # buffer: either way inside the client's own arena, so even the
                    # REPORT policy, which lets the access through, stays in owned memory
                    r = c["ranges"]
                    prot = np.flatnonzero(r.kind != 0)
                    tbytes = s["bytes"] if s["op"] == "gather" else 4 * syn.HIST_BINS
                    hole = c["buf"][target_name] + (tbytes + 255) // 256 * 256 + 64
                    dest = int(r.base[prot[0]]) if len(prot) else hole
                    bad = (dest - c["buf"][target_name]) // 4
                idx = syn.client_indices(s, n, seed, frac_bad, bad)
                self.view(c, "idx", torch.int64, n).copy_(torch.from_numpy(idx))
        self.reset()

    def reset(self, stream=None):
        """Zero every output (a, gather out, bins) and empty every log."""
        for i, c in enumerate(self.clients):
            s, n = c["spec"], c["n"]
            if s["op"] == "copy":
                self.view(c, "a", torch.float32, n).zero_()
            elif s["op"] == "gather":
                self.view(c, "out", torch.float32, n).zero_()
            else:
                self.view(c, "bins", torch.int32, syn.HIST_BINS).zero_()
            abi.agile_violation_log_init(self.log(i), i, stream)

    def log(self, i):
        return self.logs[i * abi.LOG_BYTES:(i + 1) * abi.LOG_BYTES]

    # ------------------------------------------------------------------ work

    def work(self, variant=0, guarded=True):
        items = []
        for i, c in enumerate(self.clients):
            s, b, n = c["spec"], c["buf"], c["n"]
            dev = c["dev"][variant] if guarded else None
            if s["op"] == "copy":
                w = abi.make_work("copy", dev, b["a"], b["b"], None, n, 3.0, self.policy,
                                  self.log(i), i)
            elif s["op"] == "gather":
                w = abi.make_work("gather", dev, b["out"], b["idx"], b["t"], n, 0.0, self.policy,
                                  self.log(i), i)
            else:
                w = abi.make_work("hist", dev, None, b["idx"], b["bins"], n, 0.0, self.policy,
                                  self.log(i), i)
            items.append(w)
        return items

    def run_single(self, i, variant=0, guarded=True, stream=None):
        """The client's kernel as its own launch."""
        c = self.clients[i]
        s, b, n = c["spec"], c["buf"], c["n"]
        dev = c["dev"][variant] if guarded else None
        if s["op"] == "copy":
            abi.agile_stream_launch("copy", dev, b["a"], b["b"], None, n, 3.0, self.policy,
                                    self.log(i) if guarded else None, stream)
        elif s["op"] == "gather":
            abi.agile_irregular_launch("gather", dev, b["idx"], b["t"], b["out"], n, self.policy,
                                       self.log(i) if guarded else None, stream)
        else:
            abi.agile_irregular_launch("hist", dev, b["idx"], b["bins"], None, n, self.policy,
                                       self.log(i) if guarded else None, stream)

    def outputs(self):
        """Host copies of every client's output and decoded log."""
        res = []
        for i, c in enumerate(self.clients):
            s, n = c["spec"], c["n"]
            if s["op"] == "copy":
                o = self.view(c, "a", torch.float32, n)
            elif s["op"] == "gather":
                o = self.view(c, "out", torch.float32, n)
            else:
                o = self.view(c, "bins", torch.int32, syn.HIST_BINS)
            res.append((o.cpu().numpy().copy(), abi.agile_violation_log_read(self.log(i))[1]))
        return res

    def algorithmic_bytes(self):
        """Bytes each client's kernel must move: copy 8 B/element, gather 16 B/element
        (8 index + 4 read + 4 write), histogram 8 B/element (index) plus its atomics."""
        per = {"copy": 8, "gather": 16, "hist": 8}
        return sum(per[c["spec"]["op"]] * c["n"] for c in self.clients)
