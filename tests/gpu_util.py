"""Shared helpers for the GPU tests: device buffers, table upload, oracle comparison."""
import numpy as np
import torch

import paper_2606_06697_b300 as ag

DEV = "cuda:0"


def device_table(ranges, log2_page=21, stream=None):
    """Build + upload; returns (Table, DevTable)."""
    t = ag.agile_guard_table_build(ranges.base, ranges.size, ranges.kind, ranges.ident, log2_page)
    buf = torch.empty(t.device_bytes(), dtype=torch.uint8, device=DEV)
    dev = t.upload(buf, stream)
    return t, dev


def new_log(client=0):
    log = torch.empty(ag.LOG_BYTES, dtype=torch.uint8, device=DEV)
    ag.agile_violation_log_init(log, client)
    return log


def to_dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def assert_log_equal(rec, olog, client=0):
    """Device record vs oracle Log: every field."""
    assert rec.count == olog.count, (rec, olog)
    assert rec.client == client and rec.status == 0
    if olog.count:
        assert (rec.key, rec.addr, rec.width, rec.verdict, rec.site, rec.range_id) == \
            (olog.key, olog.addr, olog.width, olog.verdict, olog.site, olog.range_id), (rec, olog)
