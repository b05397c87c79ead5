"""Kernel memory guard for B300 (sm_103a): Python binding of ``libagileguard.so``.

Argument marshalling only. Every step of the guard runs in the C/CUDA library; PyTorch
supplies device memory and streams. The names match the C entry points declared in
``include/agile_guard.h``. Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

from .abi import (  # noqa: F401
    Completion, Request, Worker, WorkerConfig, agile_worker_device_bytes,
    Graph, Work, agile_batch_autotune, agile_batch_launch_static, BATCH_STATIC_MAX_ITEMS, agile_batch_device_bytes, agile_batch_graph_create,
    agile_batch_launch, agile_batch_upload, make_work, WORK,
    AgileError, DevTable, Module, Table, ViolationRecord, agile_free, agile_guard_check_batch,
    agile_aperture_check_batch, agile_stream_launch_host, agile_selftest_bounded_waits,
    agile_guard_instrument_ptx, agile_guard_table_build, agile_irregular_launch, agile_module_bind, agile_module_launch,
    agile_irregular_launch_fastpath, agile_stream_launch_shape, FAST_PATHS,
    agile_module_load, agile_module_unload, agile_stream_launch, agile_strerror,
    agile_validate_args, agile_validate_dma, agile_version, agile_violation_log_init, agile_violation_log_read, lib,
    agile_violation_list_attach, agile_violation_list_read, list_bytes,
    library_path, LOG_BYTES, NO_RANGE, VERDICTS, KINDS, POLICIES, OPS, IRREGULAR)
