"""Failure detection without a GPU fault: the kernels' bounded waits give up on a barrier
no copy completes and on a flag nothing sets, report TIMEOUT through the log, and leave
the context usable for the next guarded launch."""
import numpy as np
import pytest
import torch

import agile_synth as syn
import oracle
import paper_2606_06697_b300 as ag
from gpu_util import DEV, device_table, new_log

pytestmark = pytest.mark.gpu


def test_bounded_waits_report_timeout_and_context_survives():
    log = new_log(client=21)
    flag = torch.zeros(4, dtype=torch.int32, device=DEV)
    res = torch.full((4,), -1, dtype=torch.int32, device=DEV)
    ag.agile_selftest_bounded_waits(log, flag, 20_000, res)
    rc, rec = ag.agile_violation_log_read(log)
    assert rc == -10 and rec.status == 1 and rec.client == 21   # AGILE_ERR_TIMEOUT
    assert int(res[0]) == 3                             # both waits gave up
    # the next guarded launch on the same context runs normally
    t = syn.table1_apertures()
    addr = np.array([0xF8000000000, 0xF0000000000], dtype=np.uint64)
    width = np.array([8, 4], dtype=np.uint8)
    _, dev = device_table(t, 21)
    d_a = torch.from_numpy(addr.view(np.int64)).to(DEV)
    d_w = torch.from_numpy(width).to(DEV)
    d_v = torch.empty(2, dtype=torch.uint8, device=DEV)
    log2 = new_log()
    ag.agile_guard_check_batch(dev, d_a, d_w, 2, d_v, log2)
    rc, rec = ag.agile_violation_log_read(log2)
    ov, _, olog = oracle.check_batch(t, addr, width)
    assert (d_v.cpu().numpy() == ov).all() and rc == 1 and rec.count == olog.count == 1


def test_flag_wait_ends_when_set():
    log = new_log()
    flag = torch.ones(4, dtype=torch.int32, device=DEV)
    res = torch.full((4,), -1, dtype=torch.int32, device=DEV)
    ag.agile_selftest_bounded_waits(log, flag, 1_000_000, res)
    torch.cuda.synchronize()
    assert int(res[0]) == 1                             # only the barrier gave up
