"""Thin ctypes binding of the C ABI in include/gx.h (argument marshalling only).

Every step of the execution path runs in the native library `_build/libgx.so`: the
verifier, the decoder and the CUDA kernels.  Importing this module fails loudly when the
library is missing; there is no fallback implementation.

Device buffers are passed as torch CUDA tensors (their data_ptr) or raw integer
addresses; streams as torch.cuda.Stream or None (legacy default stream).
"""
from __future__ import annotations

import ctypes
import os
import tempfile
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _build

OK = 0
ENOENT, E2BIG, EAGAIN, ENOMEM, EFAULT, EEXIST, EINVAL, ENOSPC = -2, -7, -11, -12, -14, -17, -22, -28
E_VERIFY, E_CUDA, E_BUDGET, E_TIMEOUT, E_DEVICE, E_ADMISSION, E_NODEV = -1000, -1001, -1002, -1003, -1004, -1005, -1006
E_FAULT = -1007  # a checked program's access outside its regions was stopped
MAP_HASH, MAP_ARRAY, MAP_RINGBUF = 1, 2, 27
ANY, NOEXIST, EXIST = 0, 1, 2

u8p = ctypes.c_void_p
u32, u64, i32, i64, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, ctypes.c_double


class MapSpec(ctypes.Structure):
    _fields_ = [("type", u32), ("key_size", u32), ("value_size", u32), ("max_entries", u32), ("flags", u32),
                ("reserved", u32)]


MAP_F_NO_DELETE = 1


def _specs(map_specs: Sequence[dict]):
    return (MapSpec * max(1, len(map_specs)))(*[MapSpec(s["type"], s["key_size"], s["value_size"], s["max_entries"],
                                                        s.get("flags", 0), 0) for s in map_specs])


class ProgOpts(ctypes.Structure):
    _fields_ = [("ctx_size", u32), ("deterministic", u32), ("insn_budget", u64), ("flags", u32), ("reserved", u32)]


class Launch(ctypes.Structure):
    _fields_ = [("block", u32), ("ept", u32), ("grid", u32), ("shards", u32), ("variant", u32), ("reserved", u32)]


class Analysis(ctypes.Structure):
    _fields_ = [("insns_processed", u64), ("stack_depth", u32), ("combinable_maps", u32)]


class SimtSpec(ctypes.Structure):
    _fields_ = [("uniform", ctypes.c_void_p), ("max_insns", u32), ("max_helper_calls", u32), ("max_mem_ops", u32),
                ("reserved", u32)]


class SimtReport(ctypes.Structure):
    _fields_ = [("max_insns", u64), ("max_helper_calls", u32), ("max_mem_ops", u32), ("uniform_branches", u32),
                ("varying_insns", u32), ("violation_pc", i32), ("violation", u32)]


# gx_simt_report.violation
(SIMT_V_NONE, SIMT_V_VERIFY, SIMT_V_BRANCH, SIMT_V_KEY, SIMT_V_ATOMIC, SIMT_V_STORE, SIMT_V_HELPER, SIMT_V_RET,
 SIMT_V_INSNS, SIMT_V_HELPERS, SIMT_V_MEM) = range(11)


# scheduling programs (gx_batch_set_sched): context layout, default hook budget, per-block tallies
SCHED_CTX = 32
SCHED_OFF_BLOCK, SCHED_OFF_SM, SCHED_OFF_DONE, SCHED_OFF_LEFT, SCHED_OFF_ELAPSED, SCHED_OFF_BUDGET = 0, 4, 8, 12, 16, 24
SCHED_MAX_INSNS, SCHED_MAX_HELPERS, SCHED_MAX_MEM = 64, 2, 16
STEAL_OWNED, STEAL_STOLEN, STEAL_ASKED, STEAL_GRANTED = range(4)
STEAL_WORDS = 4
SCHED_F_LAUNCH_CONTROL = 1


SHARDS_OFF = 255
SHARDS_AGG = 0x100  # OR into a width: warp-aggregate the updates that miss the combining cache


VARIANT_WIDE, VARIANT_CAPPED = 1, 2
GRID_PER_CHUNK = 0xFFFFFFFF  # gx_launch.grid: one block per chunk of block * ept events


def _launch(launch) -> Optional[Launch]:
    """(block, ept[, shards[, variant[, grid]]]) -> gx_launch; 0 fields mean tuned/default
    (grid 0: one wave of blocks looping over chunks; GRID_PER_CHUNK: one block per chunk)."""
    if launch is None:
        return None
    return Launch(launch[0], launch[1], launch[4] if len(launch) > 4 else 0, launch[2] if len(launch) > 2 else 0,
                  launch[3] if len(launch) > 3 else 0, 0)


class RunStats(ctypes.Structure):
    _fields_ = [("status", i32), ("fault_pc", u32), ("budget_trips", u64), ("waits_expired", u64),
                ("launches", u64)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget", u64), ("max_inflight", u32), ("max_items", u32), ("block", u32), ("ept", u32),
                ("plain", u32), ("n_progs", u32), ("progs", ctypes.POINTER(ctypes.c_void_p))]


class Completion(ctypes.Structure):
    _fields_ = [("tag", u64), ("status", i32), ("reserved", u32), ("t_arrival", dbl), ("t_start", dbl),
                ("t_done", dbl)]


class Request(ctypes.Structure):
    _fields_ = [("prog", ctypes.c_void_p), ("events_dev", ctypes.c_void_p), ("n", u64), ("ret_out_dev", ctypes.c_void_p),
                ("tag", u64), ("t_offset", dbl)]


_SIGS = {
    "gx_init": (i32, [i32, u64, ctypes.POINTER(ctypes.c_void_p)]),
    "gx_shutdown": (i32, [ctypes.c_void_p]),
    "gx_mem_used": (u64, [ctypes.c_void_p]),
    "gx_strerror": (ctypes.c_char_p, [i32]),
    "gx_map_create": (i32, [ctypes.c_void_p, u32, u32, u32, u32, u32, ctypes.POINTER(ctypes.c_void_p)]),
    "gx_map_destroy": (i32, [ctypes.c_void_p]),
    "gx_map_bytes": (u64, [ctypes.c_void_p]),
    "gx_map_read": (i32, [ctypes.c_void_p, ctypes.c_void_p, u64, ctypes.POINTER(u64), ctypes.c_void_p]),
    "gx_map_read_noalloc": (i32, [ctypes.c_void_p, ctypes.c_void_p, u64, ctypes.POINTER(u64), ctypes.c_void_p]),
    "gx_map_write": (i32, [ctypes.c_void_p, ctypes.c_void_p, u64, ctypes.c_void_p]),
    "gx_map_clear": (i32, [ctypes.c_void_p, ctypes.c_void_p]),
    "gx_ringbuf_drain": (i32, [ctypes.c_void_p, ctypes.c_void_p, u64, ctypes.POINTER(u64), ctypes.POINTER(u64),
                               ctypes.c_void_p]),
    "gx_verify": (i32, [ctypes.c_void_p, u32, ctypes.POINTER(MapSpec), u32, ctypes.POINTER(ProgOpts),
                        ctypes.c_char_p, ctypes.c_size_t]),
    "gx_analyze": (i32, [ctypes.c_void_p, u32, ctypes.POINTER(MapSpec), u32, ctypes.POINTER(ProgOpts),
                         ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    "gx_jit_check": (i32, [ctypes.c_void_p, u32, ctypes.POINTER(MapSpec), u32, ctypes.POINTER(ProgOpts),
                           ctypes.c_char_p, ctypes.c_size_t]),
    "gx_verify_simt": (i32, [ctypes.c_void_p, u32, ctypes.POINTER(MapSpec), u32, ctypes.POINTER(ProgOpts),
                             ctypes.POINTER(SimtSpec), ctypes.POINTER(SimtReport), ctypes.c_char_p, ctypes.c_size_t]),
    "gx_jit_check_simt": (i32, [ctypes.c_void_p, u32, ctypes.POINTER(MapSpec), u32, ctypes.POINTER(ProgOpts),
                                ctypes.POINTER(SimtSpec), ctypes.c_char_p, ctypes.c_size_t]),
    "gx_jit_check_sched": (i32, [ctypes.c_void_p, u32, ctypes.POINTER(MapSpec), u32, ctypes.POINTER(ProgOpts),
                                 ctypes.c_void_p, u32, ctypes.POINTER(MapSpec), u32, ctypes.POINTER(ProgOpts),
                                 ctypes.POINTER(SimtSpec), ctypes.c_char_p, ctypes.c_size_t]),
    "gx_merge_ops": (i32, [ctypes.c_void_p, u32, ctypes.POINTER(MapSpec), u32, ctypes.POINTER(ProgOpts), u32,
                           ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(u32), ctypes.c_char_p, ctypes.c_size_t]),
    "gx_verify_load": (i32, [ctypes.c_void_p, ctypes.c_void_p, u32, ctypes.POINTER(ctypes.c_void_p), u32,
                             ctypes.POINTER(ProgOpts), ctypes.POINTER(ctypes.c_void_p), ctypes.c_char_p,
                             ctypes.c_size_t]),
    "gx_verify_load_simt": (i32, [ctypes.c_void_p, ctypes.c_void_p, u32, ctypes.POINTER(ctypes.c_void_p), u32,
                                  ctypes.POINTER(ProgOpts), ctypes.POINTER(SimtSpec), ctypes.POINTER(ctypes.c_void_p),
                                  ctypes.c_char_p, ctypes.c_size_t]),
    "gx_prog_destroy": (i32, [ctypes.c_void_p]),
    "gx_prog_uops": (u32, [ctypes.c_void_p]),
    "gx_run_batch": (i32, [ctypes.c_void_p, ctypes.c_void_p, u64, ctypes.c_void_p]),
    "gx_run_batch_ex": (i32, [ctypes.c_void_p, ctypes.c_void_p, u64, u64, ctypes.c_void_p, ctypes.POINTER(Launch),
                              ctypes.c_void_p]),
    "gx_run_batch_host": (i32, [ctypes.c_void_p, ctypes.c_void_p, u64, ctypes.c_void_p]),
    "gx_last_status": (i32, [ctypes.c_void_p, ctypes.POINTER(RunStats), i32, ctypes.c_void_p]),
    "gx_autotune": (i32, [ctypes.c_void_p, ctypes.c_void_p, u64, ctypes.c_void_p, ctypes.POINTER(Launch)]),
    "gx_batch_create": (i32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "gx_batch_add": (i32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, u64, ctypes.c_void_p]),
    "gx_batch_plan": (i32, [ctypes.c_void_p, ctypes.POINTER(Launch), ctypes.c_void_p]),
    "gx_batch_launch": (i32, [ctypes.c_void_p, ctypes.c_void_p]),
    "gx_batch_destroy": (i32, [ctypes.c_void_p]),
    "gx_batch_set_sched": (i32, [ctypes.c_void_p, ctypes.c_void_p, u64, ctypes.POINTER(SimtSpec), u32,
                                 ctypes.c_char_p, ctypes.c_size_t]),
    "gx_batch_sched_tally": (i32, [ctypes.c_void_p, ctypes.c_void_p, u32, ctypes.POINTER(u32), ctypes.c_void_p]),
    "gx_server_create": (i32, [ctypes.c_void_p, ctypes.POINTER(ServerOpts), ctypes.POINTER(ctypes.c_void_p)]),
    "gx_server_submit": (i32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, u64, ctypes.c_void_p, u64, dbl]),
    "gx_server_replay": (i32, [ctypes.c_void_p, ctypes.POINTER(Request), u32, dbl]),
    "gx_server_poll": (i32, [ctypes.c_void_p, ctypes.POINTER(Completion), u32, ctypes.POINTER(u32), i32]),
    "gx_server_destroy": (i32, [ctypes.c_void_p]),
    "gx_now": (dbl, []),
}

_lib: Optional[ctypes.CDLL] = None


def default_jit_cache() -> str:
    """Where compiled programs are cached on disk unless GX_JIT_CACHE says otherwise:
    $XDG_CACHE_HOME/gx-jit, else a per-user folder under the system temporary directory.
    Never inside the package tree, so the source tree stays small whatever is compiled."""
    base = os.environ.get("XDG_CACHE_HOME")
    if base:
        return os.path.join(base, "gx-jit")
    return os.path.join(tempfile.gettempdir(), f"gx-jit-{os.getuid()}")


def lib() -> ctypes.CDLL:
    """Load the native library (building it first if it is absent or stale)."""
    global _lib
    if _lib is None:
        os.environ.setdefault("GX_JIT_CACHE", default_jit_cache())
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> List[str]:
    return list(_SIGS)


class GxError(RuntimeError):
    def __init__(self, status: int, what: str = "", log: str = "") -> None:
        msg = lib().gx_strerror(status).decode()
        super().__init__(f"{what}: {msg} ({status})" + (f": {log}" if log else ""))
        self.status = status
        self.log = log


def check(rc: int, what: str = "") -> int:
    if rc != 0:
        raise GxError(rc, what)
    return rc


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> Optional[int]:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def now() -> float:
    return lib().gx_now()


def verify(insns: np.ndarray, map_specs: Sequence[dict], ctx_size: int, deterministic: bool = False,
           insn_budget: int = 0) -> Tuple[int, str]:
    """Host-only verification: (status, log)."""
    insns = np.ascontiguousarray(insns, dtype=np.uint64)
    specs = _specs(map_specs)
    opts = ProgOpts(ctx_size, int(deterministic), insn_budget, 0, 0)
    log = ctypes.create_string_buffer(1024)
    rc = lib().gx_verify(insns.ctypes.data, insns.size, specs, len(map_specs), ctypes.byref(opts), log, 1024)
    return rc, log.value.decode()


def analyze(insns: np.ndarray, map_specs: Sequence[dict], ctx_size: int, deterministic: bool = False,
            insn_budget: int = 0) -> Tuple[int, Analysis, str]:
    """Host-only verification plus what it proved: (status, gx_analysis, log)."""
    insns = np.ascontiguousarray(insns, dtype=np.uint64)
    specs = _specs(map_specs)
    opts = ProgOpts(ctx_size, int(deterministic), insn_budget, 0, 0)
    out = Analysis()
    log = ctypes.create_string_buffer(1024)
    rc = lib().gx_analyze(insns.ctypes.data, insns.size, specs, len(map_specs), ctypes.byref(opts),
                          ctypes.byref(out), log, 1024)
    return rc, out, log.value.decode()


def verify_simt(insns: np.ndarray, map_specs: Sequence[dict], ctx_size: int, uniform=None, *, max_insns: int = 0,
                max_helper_calls: int = 0, max_mem_ops: int = 0, deterministic: bool = False,
                insn_budget: int = 0) -> Tuple[int, SimtReport, str]:
    """Host-only SIMT-aware verification (gx_verify_simt): (status, gx_simt_report, log).

    uniform: ctx_size flags marking the warp-uniform ctx bytes (None: no byte is uniform)."""
    insns = np.ascontiguousarray(insns, dtype=np.uint64)
    specs = _specs(map_specs)
    opts = ProgOpts(ctx_size, int(deterministic), insn_budget, 0, 0)
    spec, keep = _simt_spec(ctx_size, uniform, max_insns, max_helper_calls, max_mem_ops)
    out = SimtReport()
    log = ctypes.create_string_buffer(1024)
    rc = lib().gx_verify_simt(insns.ctypes.data, insns.size, specs, len(map_specs), ctypes.byref(opts),
                              ctypes.byref(spec), ctypes.byref(out), log, 1024)
    del keep
    return rc, out, log.value.decode()


def _simt_spec(ctx_size: int, uniform, max_insns: int, max_helper_calls: int, max_mem_ops: int):
    uni = None
    if uniform is not None:
        uni = np.ascontiguousarray(np.asarray(uniform, dtype=bool).astype(np.uint8))
        if uni.size != ctx_size:
            raise ValueError(f"uniform has {uni.size} flags for a {ctx_size}-byte ctx")
    return SimtSpec(None if uni is None else uni.ctypes.data, max_insns, max_helper_calls, max_mem_ops, 0), uni


def jit_check_simt(insns: np.ndarray, map_specs: Sequence[dict], ctx_size: int, uniform=None, *,
                   max_insns: int = 0, max_helper_calls: int = 0, max_mem_ops: int = 0,
                   insn_budget: int = 0) -> Tuple[int, str]:
    """Host-only: SIMT-verify and compile the warp-level form (gx_jit_check_simt): (status, log)."""
    insns = np.ascontiguousarray(insns, dtype=np.uint64)
    specs = _specs(map_specs)
    opts = ProgOpts(ctx_size, 0, insn_budget, 0, 0)
    spec, keep = _simt_spec(ctx_size, uniform, max_insns, max_helper_calls, max_mem_ops)
    log = ctypes.create_string_buffer(1 << 20)
    rc = lib().gx_jit_check_simt(insns.ctypes.data, insns.size, specs, len(map_specs), ctypes.byref(opts),
                                 ctypes.byref(spec), log, 1 << 20)
    del keep
    return rc, log.value.decode()


def _sched_limits(max_insns: Optional[int], max_helper_calls: Optional[int], max_mem_ops: Optional[int]):
    """A hook budget, or None for the library's default (GX_SCHED_MAX_*)."""
    if max_insns is None and max_helper_calls is None and max_mem_ops is None:
        return None
    return SimtSpec(None, SCHED_MAX_INSNS if max_insns is None else max_insns,
                    SCHED_MAX_HELPERS if max_helper_calls is None else max_helper_calls,
                    SCHED_MAX_MEM if max_mem_ops is None else max_mem_ops, 0)


def jit_check_sched(insns: np.ndarray, map_specs: Sequence[dict], ctx_size: int, hook: np.ndarray,
                    hook_specs: Sequence[dict], *, deterministic: bool = False, max_insns: Optional[int] = None,
                    max_helper_calls: Optional[int] = None, max_mem_ops: Optional[int] = None) -> Tuple[int, str]:
    """Host-only (gx_jit_check_sched): compile the work-stealing batch kernel of one program
    steered by the scheduling program `hook`: (status, log)."""
    insns = np.ascontiguousarray(insns, dtype=np.uint64)
    hook = np.ascontiguousarray(hook, dtype=np.uint64)
    specs, hspecs = _specs(map_specs), _specs(hook_specs)
    opts = ProgOpts(ctx_size, int(deterministic), 0, 0, 0)
    hopts = ProgOpts(SCHED_CTX, 0, 0, 0, 0)
    lim = _sched_limits(max_insns, max_helper_calls, max_mem_ops)
    log = ctypes.create_string_buffer(1 << 20)
    rc = lib().gx_jit_check_sched(insns.ctypes.data, insns.size, specs, len(map_specs), ctypes.byref(opts),
                                  hook.ctypes.data, hook.size, hspecs, len(hook_specs), ctypes.byref(hopts),
                                  None if lim is None else ctypes.byref(lim), log, 1 << 20)
    return rc, log.value.decode()


# gx_merge_ops word codes
MERGE_NONE, MERGE_ADD, MERGE_OR, MERGE_AND, MERGE_XOR, MERGE_MAX, MERGE_MIN = range(7)
MERGE_W8 = 0x10


def merge_ops(insns: np.ndarray, map_specs: Sequence[dict], ctx_size: int, map_index: int,
              insn_budget: int = 0) -> Tuple[int, np.ndarray, Optional[bytes], str]:
    """Host-only (gx_merge_ops): (status, per-4-byte-word merge codes, the hash insert's constant
    bytes or None when the program never inserts, log)."""
    insns = np.ascontiguousarray(insns, dtype=np.uint64)
    specs = _specs(map_specs)
    opts = ProgOpts(ctx_size, 1, insn_budget, 0, 0)
    vs = int(map_specs[map_index]["value_size"]) if 0 <= map_index < len(map_specs) else 0
    ops = np.zeros(max(1, (vs + 3) // 4), dtype=np.uint8)
    ins = np.zeros(max(1, vs), dtype=np.uint8)
    has = u32(0)
    log = ctypes.create_string_buffer(1024)
    rc = lib().gx_merge_ops(insns.ctypes.data, insns.size, specs, len(map_specs), ctypes.byref(opts), map_index,
                            ops.ctypes.data, ins.ctypes.data, ctypes.byref(has), log, 1024)
    return rc, ops[:(vs + 3) // 4], (ins[:vs].tobytes() if has.value else None), log.value.decode()


PROG_JIT = 1
PROG_CHECKED = 2  # the checked interpreter: every access tested against the event's regions


def jit_check(insns: np.ndarray, map_specs: Sequence[dict], ctx_size: int, deterministic: bool = False,
              insn_budget: int = 0) -> Tuple[int, str]:
    """Host-only: verify and compile the specialised form (no device): (status, log)."""
    insns = np.ascontiguousarray(insns, dtype=np.uint64)
    specs = _specs(map_specs)
    opts = ProgOpts(ctx_size, int(deterministic), insn_budget, PROG_JIT, 0)
    log = ctypes.create_string_buffer(8192)
    rc = lib().gx_jit_check(insns.ctypes.data, insns.size, specs, len(map_specs), ctypes.byref(opts), log, 8192)
    return rc, log.value.decode()


def precompile(programs: Sequence[Tuple], deterministic: bool = True, threads: Optional[int] = None) -> List[int]:
    """Host-only: compile the specialised form of many programs at once, one host thread per
    program (gx_jit_check each), so that loading them afterwards reads the disk cache
    (GX_JIT_CACHE) instead of compiling one after another.  `programs` holds
    (insns, map specs, ctx_size) triples; returns each one's status."""
    from concurrent.futures import ThreadPoolExecutor

    lib()
    items = list(programs)
    if not items:
        return []
    with ThreadPoolExecutor(max_workers=threads or min(len(items), os.cpu_count() or 1)) as ex:
        return [rc for rc, _ in ex.map(lambda t: jit_check(t[0], t[1], t[2], deterministic=deterministic), items)]


class Context:
    def __init__(self, device: int = 0, mem_budget: int = 0) -> None:
        h = ctypes.c_void_p()
        check(lib().gx_init(device, mem_budget, ctypes.byref(h)), "gx_init")
        self.h = h

    def mem_used(self) -> int:
        return lib().gx_mem_used(self.h)

    def close(self) -> None:
        if self.h:
            check(lib().gx_shutdown(self.h), "gx_shutdown")
            self.h = None


class Map:
    def __init__(self, ctx: Context, type: int, key_size: int, value_size: int, max_entries: int,
                 flags: int = 0) -> None:
        h = ctypes.c_void_p()
        check(lib().gx_map_create(ctx.h, type, key_size, value_size, max_entries, flags, ctypes.byref(h)),
              "gx_map_create")
        self.h, self.ctx, self.flags = h, ctx, flags
        self.type, self.key_size, self.value_size, self.max_entries = type, key_size, value_size, max_entries

    @classmethod
    def from_spec(cls, ctx: Context, spec: dict) -> "Map":
        return cls(ctx, spec["type"], spec["key_size"], spec["value_size"], spec["max_entries"],
                   flags=spec.get("flags", 0))

    def destroy(self) -> None:
        if self.h:
            check(lib().gx_map_destroy(self.h), "gx_map_destroy")
            self.h = None

    def nbytes(self) -> int:
        return lib().gx_map_bytes(self.h)

    def read_raw(self, stream=None) -> Tuple[bytes, int]:
        if self.type == MAP_ARRAY:
            cap = self.max_entries * self.value_size
        else:
            cap = self.max_entries * (self.key_size + self.value_size)
        buf = np.zeros(max(cap, 1), dtype=np.uint8)
        n = u64(0)
        check(lib().gx_map_read(self.h, buf.ctypes.data, cap, ctypes.byref(n), _stream(stream)), "gx_map_read")
        used = self.max_entries * self.value_size if self.type == MAP_ARRAY else n.value * (self.key_size + self.value_size)
        return buf[:used].tobytes(), n.value

    def array_values(self, stream=None) -> np.ndarray:
        raw, _ = self.read_raw(stream)
        return np.frombuffer(raw, dtype=np.uint8).reshape(self.max_entries, self.value_size)

    def array_u64(self, stream=None) -> np.ndarray:
        return self.array_values(stream).view("<u8").reshape(self.max_entries, self.value_size // 8)

    def hash_items(self, stream=None) -> Dict[bytes, bytes]:
        raw, n = self.read_raw(stream)
        st = self.key_size + self.value_size
        return {raw[i * st:i * st + self.key_size]: raw[i * st + self.key_size:(i + 1) * st] for i in range(n)}

    def write(self, data: bytes, stream=None) -> None:
        buf = np.frombuffer(data, dtype=np.uint8).copy()
        check(lib().gx_map_write(self.h, buf.ctypes.data, buf.size, _stream(stream)), "gx_map_write")

    def clear(self, stream=None) -> None:
        check(lib().gx_map_clear(self.h, _stream(stream)), "gx_map_clear")

    def drain(self, stream=None) -> Tuple[bytes, int]:
        """Ring buffer: (packed committed records, drops since the last drain)."""
        buf = np.zeros(self.max_entries, dtype=np.uint8)
        nb, dropped = u64(0), u64(0)
        check(lib().gx_ringbuf_drain(self.h, buf.ctypes.data, buf.size, ctypes.byref(nb), ctypes.byref(dropped),
                                     _stream(stream)), "gx_ringbuf_drain")
        return buf[:nb.value].tobytes(), dropped.value


class Program:
    def __init__(self, ctx: Context, insns: np.ndarray, maps: Sequence[Map], ctx_size: int,
                 deterministic: bool = False, insn_budget: int = 0, jit: bool = False,
                 simt: Optional[dict] = None, checked: bool = False) -> None:
        """simt: load the warp-level form (gx_verify_load_simt) with these gx_simt_spec fields:
        uniform (ctx_size flags) and optionally max_insns, max_helper_calls, max_mem_ops;
        it needs jit=True.  checked: run through the checked interpreter (GX_PROG_CHECKED)."""
        insns = np.ascontiguousarray(insns, dtype=np.uint64)
        arr = (ctypes.c_void_p * max(1, len(maps)))(*[m.h for m in maps])
        opts = ProgOpts(ctx_size, int(deterministic), insn_budget, (PROG_JIT if jit else 0) | (PROG_CHECKED if checked else 0),
                        0)
        log = ctypes.create_string_buffer(8192)
        h = ctypes.c_void_p()
        if simt is None:
            rc = lib().gx_verify_load(ctx.h, insns.ctypes.data, insns.size, arr, len(maps), ctypes.byref(opts),
                                      ctypes.byref(h), log, 8192)
        else:
            spec, keep = _simt_spec(ctx_size, simt.get("uniform"), simt.get("max_insns", 0),
                                    simt.get("max_helper_calls", 0), simt.get("max_mem_ops", 0))
            rc = lib().gx_verify_load_simt(ctx.h, insns.ctypes.data, insns.size, arr, len(maps), ctypes.byref(opts),
                                           ctypes.byref(spec), ctypes.byref(h), log, 8192)
            del keep
        if rc:
            raise GxError(rc, "gx_verify_load" if simt is None else "gx_verify_load_simt", log.value.decode())
        self.h, self.ctx, self.maps, self.ctx_size = h, ctx, list(maps), ctx_size

    def destroy(self) -> None:
        if self.h:
            check(lib().gx_prog_destroy(self.h), "gx_prog_destroy")
            self.h = None

    def uops(self) -> int:
        return lib().gx_prog_uops(self.h)

    def run(self, events, n: Optional[int] = None, *, ret_out=None, idx_base: int = 0,
            launch: Optional[Tuple[int, ...]] = None, stream=None) -> None:
        if n is None:
            n = events.numel() * events.element_size() // self.ctx_size
        lp = None if launch is None else ctypes.byref(_launch(launch))
        check(lib().gx_run_batch_ex(self.h, _ptr(events), n, idx_base, _ptr(ret_out), lp, _stream(stream)),
              "gx_run_batch_ex")

    def run_host(self, events_host: np.ndarray, ret_out_host: Optional[np.ndarray] = None) -> None:
        raw = events_host.view(np.uint8).reshape(-1)
        n = raw.size // self.ctx_size
        check(lib().gx_run_batch_host(self.h, raw.ctypes.data, n, _ptr(ret_out_host)), "gx_run_batch_host")

    def status(self, reset: bool = False, stream=None) -> RunStats:
        st = RunStats()
        check(lib().gx_last_status(self.h, ctypes.byref(st), int(reset), _stream(stream)), "gx_last_status")
        return st

    def autotune(self, events, n: Optional[int] = None, stream=None) -> Tuple[int, int, int]:
        """Returns the chosen (block, ept, shards); the kernel variant is in self.tuned_variant and
        the grid choice (0 = one wave, GRID_PER_CHUNK) in self.tuned_grid."""
        if n is None:
            n = events.numel() * events.element_size() // self.ctx_size
        best = Launch()
        check(lib().gx_autotune(self.h, _ptr(events), n, _stream(stream), ctypes.byref(best)), "gx_autotune")
        self.tuned_variant = best.variant
        self.tuned_grid = best.grid
        return best.block, best.ept, best.shards


class Batch:
    def __init__(self, ctx: Context) -> None:
        h = ctypes.c_void_p()
        check(lib().gx_batch_create(ctx.h, ctypes.byref(h)), "gx_batch_create")
        self.h = h

    def add(self, prog: Program, events, n: int, ret_out=None) -> None:
        check(lib().gx_batch_add(self.h, prog.h, _ptr(events), n, _ptr(ret_out)), "gx_batch_add")

    def plan(self, launch: Optional[Tuple[int, ...]] = None, stream=None) -> None:
        lp = None if launch is None else ctypes.byref(_launch(launch))
        check(lib().gx_batch_plan(self.h, lp, _stream(stream)), "gx_batch_plan")

    def launch(self, stream=None) -> None:
        check(lib().gx_batch_launch(self.h, _stream(stream)), "gx_batch_launch")

    def set_sched(self, hook: Program, budget_ns: int = 0, *, launch_control: bool = False,
                  max_insns: Optional[int] = None, max_helper_calls: Optional[int] = None,
                  max_mem_ops: Optional[int] = None) -> None:
        """Steer the blocks with a scheduling program (gx_batch_set_sched); before plan().
        launch_control: one block per chunk, stealing by cancelling blocks not yet started."""
        lim = _sched_limits(max_insns, max_helper_calls, max_mem_ops)
        log = ctypes.create_string_buffer(1 << 16)
        rc = lib().gx_batch_set_sched(self.h, hook.h, budget_ns, None if lim is None else ctypes.byref(lim),
                                      SCHED_F_LAUNCH_CONTROL if launch_control else 0, log, 1 << 16)
        check(rc, "gx_batch_set_sched: " + log.value.decode())
        self._sched = hook

    def sched_tally(self, stream=None) -> np.ndarray:
        """The last launch's per-block counters (gx_batch_sched_tally): uint32 [blocks, STEAL_WORDS]."""
        n = u32(0)
        rc = lib().gx_batch_sched_tally(self.h, None, 0, ctypes.byref(n), _stream(stream))
        if rc not in (OK, ENOSPC):
            check(rc, "gx_batch_sched_tally")
        out = np.zeros((max(1, n.value), STEAL_WORDS), dtype=np.uint32)
        check(lib().gx_batch_sched_tally(self.h, out.ctypes.data, n.value, ctypes.byref(n), _stream(stream)),
              "gx_batch_sched_tally")
        return out[:n.value]

    def destroy(self) -> None:
        if self.h:
            check(lib().gx_batch_destroy(self.h), "gx_batch_destroy")
            self.h = None


class Server:
    def __init__(self, ctx: Context, mem_budget: int = 0, max_inflight: int = 2, max_items: int = 1024,
                 block: int = 256, ept: int = 4, plain: bool = False, progs: Sequence["Program"] = ()) -> None:
        self._progs = (ctypes.c_void_p * max(1, len(progs)))(*[p.h for p in progs])
        opts = ServerOpts(mem_budget, max_inflight, max_items, block, ept, int(plain), len(progs), self._progs)
        h = ctypes.c_void_p()
        check(lib().gx_server_create(ctx.h, ctypes.byref(opts), ctypes.byref(h)), "gx_server_create")
        self.h = h

    def submit(self, prog: Program, events, n: int, ret_out=None, tag: int = 0, t_arrival: float = 0.0) -> None:
        check(lib().gx_server_submit(self.h, prog.h, _ptr(events), n, _ptr(ret_out), tag, t_arrival),
              "gx_server_submit")

    def replay(self, reqs: Sequence[Tuple[Program, object, int, object, int, float]], t0: float = 0.0) -> None:
        arr = (Request * len(reqs))()
        for i, (p, ev, n, ro, tag, toff) in enumerate(reqs):
            arr[i] = Request(p.h, _ptr(ev), n, _ptr(ro), tag, toff)
        check(lib().gx_server_replay(self.h, arr, len(reqs), t0), "gx_server_replay")

    def poll(self, cap: int = 4096, wait_ms: int = 0) -> List[Completion]:
        buf = (Completion * cap)()
        n = u32(0)
        check(lib().gx_server_poll(self.h, buf, cap, ctypes.byref(n), wait_ms), "gx_server_poll")
        return [buf[i] for i in range(n.value)]

    def destroy(self) -> None:
        if self.h:
            check(lib().gx_server_destroy(self.h), "gx_server_destroy")
            self.h = None


def parse_records(raw: bytes) -> List[Tuple[int, bytes]]:
    """Split a drained record stream into (event_idx, payload) in stream order."""
    out, pos = [], 0
    while pos + 16 <= len(raw):
        ln = int.from_bytes(raw[pos:pos + 4], "little")
        idx = int.from_bytes(raw[pos + 8:pos + 16], "little")
        out.append((idx, raw[pos + 16:pos + 16 + ln]))
        pos += 16 + ((ln + 7) & ~7)
    return out
