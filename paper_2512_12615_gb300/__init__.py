"""gx: a device-side eBPF execution engine for GB300 (sm_103a).

The native library (verifier, decoder, CUDA kernels, runtime) is built in-tree by
`_build.build()` and bound by `gx.py`; see include/gx.h for the C ABI.
"""
from .gx import (  # noqa: F401
    ANY, E_ADMISSION, E_BUDGET, E_CUDA, E_DEVICE, E_FAULT, E_NODEV, PROG_CHECKED, E_TIMEOUT, E_VERIFY, E2BIG, EAGAIN, EEXIST, EINVAL,
    ENOENT, ENOMEM, EXIST, MAP_ARRAY, MAP_F_NO_DELETE, MAP_HASH, MAP_RINGBUF, NOEXIST, SHARDS_AGG, SHARDS_OFF, Batch, Context, GxError, Map, Program,
    GRID_PER_CHUNK, Server, VARIANT_CAPPED, VARIANT_WIDE, analyze, check, exported_symbols, jit_check, lib, now, parse_records, precompile, verify,
    SIMT_V_ATOMIC, SIMT_V_BRANCH, SIMT_V_HELPER, SIMT_V_HELPERS, SIMT_V_INSNS, SIMT_V_KEY, SIMT_V_MEM, SIMT_V_NONE,
    SIMT_V_RET, SIMT_V_STORE, SIMT_V_VERIFY, SimtReport, jit_check_simt, verify_simt,
    MERGE_ADD, MERGE_AND, MERGE_MAX, MERGE_MIN, MERGE_NONE, MERGE_OR, MERGE_W8, MERGE_XOR, merge_ops,
    SCHED_CTX, SCHED_MAX_HELPERS, SCHED_MAX_INSNS, SCHED_MAX_MEM, SCHED_OFF_BLOCK, SCHED_OFF_BUDGET,
    SCHED_OFF_DONE, SCHED_OFF_ELAPSED, SCHED_OFF_LEFT, SCHED_OFF_SM, STEAL_ASKED, STEAL_GRANTED, STEAL_OWNED,
    STEAL_STOLEN, STEAL_WORDS, SCHED_F_LAUNCH_CONTROL, jit_check_sched,
)
from . import merge  # noqa: F401,E402
