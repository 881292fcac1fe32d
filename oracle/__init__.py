"""ORACLE -- test infrastructure only.

Python loader for the plain sequential CPU eBPF interpreter in `gx_oracle.c`.
Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may import
this package; the engine (`paper_2512_12615_gb300`) never does, and the two share no code.

A batch run follows the plain definition: events in index order, one program execution
per event on a fresh register file and stack, maps and ring buffers carried over between
events (the device handlers of Sec. 4.3 / Sec. 5.3 executed one after another; instruction
semantics from the standard eBPF ISA, RFC 9669).

`run_warps` is the warp-level form of Sec. 4.4.1 / Sec. 4.4.2: groups of up to 32
consecutive events run one handler in lockstep, lane-varying values may not decide control
flow or reach shared state, and side effects happen once per warp.  It reports where the
lanes would disagree (EDIVERGE), which is what a SIMT-aware verifier must rule out.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gx_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")

MAP_HASH, MAP_ARRAY, MAP_RINGBUF = 1, 2, 27
ENOENT, E2BIG, EAGAIN, ENOMEM, EFAULT, EEXIST, EINVAL, EBUDGET = -2, -7, -11, -12, -14, -17, -22, -1002
EDIVERGE = -1003  # run_warps: the lanes of a warp disagree where they must agree
EDEFER = -1004  # run with defer_maps: a deferred map's values were used other than by a combinable update

_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


def build(force: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fno-strict-aliasing", SRC, "-o", tmp])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_PATH)
            vp, u32, u64, i64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int
            L.or_map_create.argtypes = [u32, u32, u32, u32]
            L.or_map_create.restype = vp
            L.or_map_destroy.argtypes = [vp]
            L.or_map_update.argtypes = [vp, vp, vp, u64]
            L.or_map_update.restype = i32
            L.or_map_delete.argtypes = [vp, vp]
            L.or_map_delete.restype = i32
            L.or_map_lookup.argtypes = [vp, vp, vp]
            L.or_map_lookup.restype = i32
            L.or_array_read.argtypes = [vp, vp, u64]
            L.or_array_read.restype = i64
            L.or_hash_count.argtypes = [vp]
            L.or_hash_count.restype = i64
            L.or_hash_dump.argtypes = [vp, vp, u64]
            L.or_hash_dump.restype = i64
            L.or_ringbuf_read.argtypes = [vp, vp, u64, ctypes.POINTER(u64)]
            L.or_ringbuf_read.restype = i64
            L.or_ringbuf_reset.argtypes = [vp]
            L.or_run.argtypes = [vp, u32, vp, u32, vp, u64, u32, u64, vp, ctypes.POINTER(u64), u64,
                                 ctypes.POINTER(u64)]
            L.or_run.restype = i32
            L.or_run_flags.argtypes = L.or_run.argtypes + [u32, ctypes.POINTER(u64), u32]
            L.or_run_flags.restype = i32
            L.or_run_warps.argtypes = [vp, u32, vp, u32, vp, u64, u32, vp, u32, u64, vp, ctypes.POINTER(u64), u64,
                                       ctypes.POINTER(u64), ctypes.POINTER(u32)]
            L.or_run_warps.restype = i32
            _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, rc: int, event: int, pc: Optional[int] = None) -> None:
        where = f" at event {event}" + ("" if pc is None else f", insn {pc}")
        super().__init__(f"oracle run failed rc={rc}{where}")
        self.rc = rc
        self.event = event
        self.pc = pc


class Map:
    """One oracle map (array, hash or ring buffer)."""

    def __init__(self, type: int, key_size: int, value_size: int, max_entries: int) -> None:
        self.type, self.key_size, self.value_size, self.max_entries = type, key_size, value_size, max_entries
        self.h = lib().or_map_create(type, key_size, value_size, max_entries)
        if not self.h:
            raise ValueError(f"bad map spec {(type, key_size, value_size, max_entries)}")

    @classmethod
    def from_spec(cls, spec: dict) -> "Map":
        return cls(spec["type"], spec["key_size"], spec["value_size"], spec["max_entries"])

    def __del__(self) -> None:
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.or_map_destroy(h)
            self.h = None

    # host-side access
    def update(self, key: bytes, value: bytes, flags: int = 0) -> int:
        assert len(key) == self.key_size and len(value) == self.value_size
        return lib().or_map_update(self.h, key, value, flags)

    def delete(self, key: bytes) -> int:
        return lib().or_map_delete(self.h, key)

    def lookup(self, key: bytes) -> Optional[bytes]:
        buf = ctypes.create_string_buffer(self.value_size)
        rc = lib().or_map_lookup(self.h, key, buf)
        return None if rc else buf.raw

    def array_values(self) -> np.ndarray:
        """Raw value bytes, shape (max_entries, value_size)."""
        out = np.zeros((self.max_entries, self.value_size), dtype=np.uint8)
        rc = lib().or_array_read(self.h, out.ctypes.data, out.nbytes)
        assert rc == out.nbytes, rc
        return out

    def array_u64(self) -> np.ndarray:
        return self.array_values().view("<u8").reshape(self.max_entries, self.value_size // 8)

    def hash_items(self) -> dict:
        """{key bytes: value bytes} of the live entries."""
        n = lib().or_hash_count(self.h)
        stride = self.key_size + self.value_size
        buf = np.zeros(max(1, n) * stride, dtype=np.uint8)
        k = lib().or_hash_dump(self.h, buf.ctypes.data, n)
        assert k == n, (k, n)
        raw = buf.tobytes()
        return {raw[i * stride:i * stride + self.key_size]: raw[i * stride + self.key_size:(i + 1) * stride]
                for i in range(n)}

    def ringbuf_records(self) -> Tuple[List[Tuple[int, bytes]], int]:
        """([(event_idx, payload bytes)] in emission order, dropped count)."""
        buf = np.zeros(self.max_entries, dtype=np.uint8)
        dropped = ctypes.c_uint64(0)
        n = lib().or_ringbuf_read(self.h, buf.ctypes.data, buf.nbytes, ctypes.byref(dropped))
        assert n >= 0, n
        return parse_records(buf[:n].tobytes()), int(dropped.value)

    def ringbuf_reset(self) -> None:
        lib().or_ringbuf_reset(self.h)


def parse_records(raw: bytes) -> List[Tuple[int, bytes]]:
    """Split a packed record stream {u32 len; u32 flags; u64 event_idx; payload pad 8}."""
    out, pos = [], 0
    while pos + 16 <= len(raw):
        ln = int.from_bytes(raw[pos:pos + 4], "little")
        idx = int.from_bytes(raw[pos + 8:pos + 16], "little")
        out.append((idx, raw[pos + 16:pos + 16 + ln]))
        pos += 16 + ((ln + 7) & ~7)
    return out


def run(prog: np.ndarray, maps: Sequence[Map], events: np.ndarray, ctx_size: int, *, event_idx_base: int = 0,
        want_r0: bool = False, budget: int = 0, strict_align: bool = False,
        most: Optional[list] = None, defer_maps: int = 0) -> Tuple[Optional[np.ndarray], int]:
    """Run `prog` over `events` (contiguous records of ctx_size bytes).

    Returns (R0 per event as int64 or None, total executed instructions); raises
    OracleError on a fault.  strict_align: a load, store or atomic at an address that is
    not a multiple of its size is a fault (EFAULT) too.  most (a list, filled in): the most
    instructions, helper calls and loads / stores / atomics one event executed.  defer_maps:
    bit m defers map m's non-fetching commutative updates to after the last event; any
    other use of its values raises EDEFER (the oracle's model of block-private combining)."""
    prog = np.ascontiguousarray(prog, dtype=np.uint64)
    raw = np.ascontiguousarray(events).view(np.uint8).reshape(-1)
    assert raw.size % ctx_size == 0
    n = raw.size // ctx_size
    handles = (ctypes.c_void_p * max(1, len(maps)))(*[m.h for m in maps])
    r0 = np.zeros(n, dtype=np.int64) if want_r0 else None
    count = ctypes.c_uint64(0)
    bad = ctypes.c_uint64(0)
    top = (ctypes.c_uint64 * 3)()
    rc = lib().or_run_flags(prog.ctypes.data, prog.size, handles, len(maps), raw.ctypes.data, n, ctx_size,
                            event_idx_base, None if r0 is None else r0.ctypes.data, ctypes.byref(count), budget,
                            ctypes.byref(bad), 1 if strict_align else 0, top, defer_maps)
    if most is not None:
        most[:] = [int(x) for x in top]
    if rc != 0:
        raise OracleError(rc, int(bad.value))
    return r0, int(count.value)


def run_warps(prog: np.ndarray, maps: Sequence[Map], events: np.ndarray, ctx_size: int, *,
              uniform: Optional[np.ndarray] = None, lanes: int = 32, event_idx_base: int = 0, want_r0: bool = False,
              budget: int = 0) -> Tuple[Optional[np.ndarray], int]:
    """Run `prog` over `events` as warps of `lanes` consecutive events in lockstep.

    uniform: ctx_size booleans marking the warp-uniform ctx bytes (every lane of a warp must
    carry the same value there).  Returns (R0 per event or None, instructions per warp
    summed); raises OracleError (rc EDIVERGE where the lanes disagree, with the insn)."""
    prog = np.ascontiguousarray(prog, dtype=np.uint64)
    raw = np.ascontiguousarray(events).view(np.uint8).reshape(-1)
    assert raw.size % ctx_size == 0
    n = raw.size // ctx_size
    uni = None
    if uniform is not None:
        uni = np.ascontiguousarray(np.asarray(uniform, dtype=bool).astype(np.uint8))
        assert uni.size == ctx_size
    handles = (ctypes.c_void_p * max(1, len(maps)))(*[m.h for m in maps])
    r0 = np.zeros(n, dtype=np.int64) if want_r0 else None
    count = ctypes.c_uint64(0)
    bad = ctypes.c_uint64(0)
    pc = ctypes.c_uint32(0)
    rc = lib().or_run_warps(prog.ctypes.data, prog.size, handles, len(maps), raw.ctypes.data, n, ctx_size,
                            None if uni is None else uni.ctypes.data, lanes, event_idx_base,
                            None if r0 is None else r0.ctypes.data, ctypes.byref(count), budget, ctypes.byref(bad),
                            ctypes.byref(pc))
    if rc != 0:
        raise OracleError(rc, int(bad.value), int(pc.value))
    return r0, int(count.value)


def maps_from_specs(specs: Sequence[dict]) -> List[Map]:
    return [Map.from_spec(s) for s in specs]


# ------------------------------------------------------------------ several parts at once
def _combine(op: str, width: int, start: int, vals: List[int]) -> int:
    """One value word merged over the parts that hold it, from its starting value `start`."""
    mask = (1 << (8 * width)) - 1
    r = start
    for v in vals:
        if op == "add":
            r = (r + v - start) & mask
        elif op == "xor":
            r ^= v ^ start
        elif op == "or":
            r |= v
        elif op == "and":
            r &= v
        elif op == "max":
            r = max(r, v)
        elif op == "min":
            r = min(r, v)
        else:
            raise ValueError(op)
    return r


def _merge_value(words, free: List[int], start: bytes, vals: List[bytes]) -> bytes:
    """vals merged word by word; `free` lists the bytes no update reaches."""
    out = bytearray(vals[0])
    for v in vals[1:]:  # bytes no update reaches are the same in every part
        for b in free:
            if v[b] != out[b]:
                raise ValueError(f"byte {b} differs between parts but no update reaches it")
    for off, width, op in words:
        r = _combine(op, width, int.from_bytes(start[off:off + width], "little"),
                     [int.from_bytes(v[off:off + width], "little") for v in vals])
        out[off:off + width] = r.to_bytes(width, "little")
    return bytes(out)


def run_parallel(prog: np.ndarray, specs: Sequence[dict], events: np.ndarray, ctx_size: int, merge: Sequence,
                 *, threads: Optional[int] = None, event_idx_base: int = 0, budget: int = 0,
                 init: Optional[Sequence[Optional[bytes]]] = None) -> Tuple[list, int]:
    """`run` over `threads` contiguous parts of `events` at once, each part with maps of its
    own and its global event base, merged afterwards.  Equal to `run` over the whole batch
    when the program changes map values only by commutative updates (the deterministic
    reading of Sec. 4.4.3), which makes the parts' order irrelevant.

    merge: per map, how its values combine, from the caller's knowledge of the program:
    {"words": [(byte offset, width, op)], "insert": bytes of a new hash key} with op one of
    add, xor, or, and, max, min (None for ring buffers).  init: per array map, the starting
    contents (None = zeros).  Returns (snapshots, executed instructions): per map the
    array bytes (max_entries x value_size), the {key: value} dict, or (records, dropped)."""
    from concurrent.futures import ThreadPoolExecutor

    raw = np.ascontiguousarray(events).view(np.uint8).reshape(-1)
    n = raw.size // ctx_size
    t = max(1, min(threads or os.cpu_count() or 1, n or 1))
    cuts = [n * j // t for j in range(t + 1)]

    def part(j):
        maps = maps_from_specs(specs)
        for m, v in zip(maps, init or [None] * len(maps)):
            if v is not None:
                for k in range(m.max_entries):
                    m.update(k.to_bytes(4, "little"), v[k * m.value_size:(k + 1) * m.value_size])
        _, count = run(prog, maps, raw[cuts[j] * ctx_size:cuts[j + 1] * ctx_size], ctx_size,
                       event_idx_base=event_idx_base + cuts[j], budget=budget)
        snaps = []
        for m in maps:
            if m.type == MAP_ARRAY:
                snaps.append(m.array_values())
            elif m.type == MAP_HASH:
                snaps.append(m.hash_items())
            else:
                snaps.append(m.ringbuf_records())
        return snaps, count

    with ThreadPoolExecutor(max_workers=t) as pool:  # the C interpreter runs without the GIL
        parts = list(pool.map(part, range(t)))
    out = []
    for i, spec in enumerate(specs):
        copies = [p[0][i] for p in parts]
        if spec["type"] == MAP_RINGBUF:  # the parts are in event order and so are their records
            out.append(([r for recs, _ in copies for r in recs], sum(d for _, d in copies)))
            continue
        words = merge[i]["words"]
        free = [b for b in range(spec["value_size"]) if not any(o <= b < o + w for o, w, _ in words)]
        if spec["type"] == MAP_ARRAY:
            vs = spec["value_size"]
            start = init[i] if init and init[i] is not None else bytes(spec["max_entries"] * vs)
            arr = np.zeros((spec["max_entries"], vs), dtype=np.uint8)
            for k in range(spec["max_entries"]):
                vals = [c[k].tobytes() for c in copies]
                arr[k] = np.frombuffer(_merge_value(words, free, start[k * vs:(k + 1) * vs], vals), dtype=np.uint8)
            out.append(arr)
        else:
            merged = {}
            for key in {k for c in copies for k in c}:
                merged[key] = _merge_value(words, free, merge[i]["insert"], [c[key] for c in copies if key in c])
            out.append(merged)
    return out, sum(c for _, c in parts)
