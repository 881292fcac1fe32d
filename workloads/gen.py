"""Python side of the seeded event generator (`evgen.c`), shared by oracle and engine tests.

Records are returned as a contiguous uint8 buffer viewed through `EVENT_DTYPE`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libgxgen.so")
SRC = os.path.join(HERE, "evgen.c")

EVENT_DTYPE = np.dtype(
    [("addr", "<u8"), ("sm_id", "<u4"), ("warp_id", "<u4"), ("ts_ns", "<u8"), ("kind", "<u4"), ("size", "<u4")]
)
assert EVENT_DTYPE.itemsize == 32

BASE_SEED = 0x6758
_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


def build(force: bool = False) -> str:
    """Compile evgen.c into an in-tree shared library (plain C, no arch flags)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_PATH)
            u64, i32, vp, dbl, u32 = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_uint32
            L.evgen_uniform.argtypes = [u64, u64, vp, i32]
            L.evgen_pageheat.argtypes = [u64, u64, dbl, u32, vp, i32]
            L.evgen_latency_pairs.argtypes = [u64, u64, dbl, dbl, u32, vp, i32]
            L.evgen_warp_access.argtypes = [u64, u64, u32, dbl, u32, dbl, vp, i32]
            L.evgen_draw.argtypes = [u64, u64, u32]
            L.evgen_draw.restype = u64
            for f in (L.evgen_uniform, L.evgen_pageheat, L.evgen_latency_pairs, L.evgen_warp_access):
                f.restype = i32
            _lib = L
    return _lib


def _threads(nthreads: Optional[int]) -> int:
    return nthreads or min(64, os.cpu_count() or 1)


def _alloc(n_records: int, out: Optional[np.ndarray]) -> np.ndarray:
    if out is None:
        return np.zeros(n_records, dtype=EVENT_DTYPE)
    assert out.dtype == EVENT_DTYPE and out.size >= n_records and out.flags.c_contiguous
    return out[:n_records]


def uniform_events(n: int, seed: int = BASE_SEED, out=None, nthreads=None) -> np.ndarray:
    """addr uniform over [0, 2^32); sm_id 0..147; warp_id 0..63; ts with exp(1 us) gaps;
    kind 0..7; size in {4, 8, 16, 32}."""
    ev = _alloc(n, out)
    rc = lib().evgen_uniform(seed, n, ev.ctypes.data, _threads(nthreads))
    assert rc == 0, rc
    return ev


def pageheat_events(n: int, seed: int = BASE_SEED, s: float = 1.1, log2_pages: int = 24, out=None,
                    nthreads=None) -> np.ndarray:
    """addr = page*4096 + size-aligned offset; page Zipf(s) over 2^log2_pages 4 KiB pages
    (2^24 pages = a 64 GiB space); other fields as in `uniform_events`."""
    ev = _alloc(n, out)
    rc = lib().evgen_pageheat(seed, n, s, log2_pages, ev.ctypes.data, _threads(nthreads))
    assert rc == 0, rc
    return ev


def warp_access_events(n_warps: int, seed: int = BASE_SEED, lanes: int = 32, s: float = 1.1, log2_pages: int = 24,
                       coalesced: float = 0.75, out=None, nthreads=None) -> np.ndarray:
    """n_warps * lanes records, one warp-context memory access per warp: the lanes of warp w
    (records w*lanes ..) share sm_id, warp_id, ts_ns, kind and size; a fraction `coalesced`
    of the warps access consecutive size-strided addresses from one Zipf(s) page, the
    others one Zipf(s) page per lane."""
    ev = _alloc(n_warps * lanes, out)
    rc = lib().evgen_warp_access(seed, n_warps, lanes, s, log2_pages, coalesced, ev.ctypes.data, _threads(nthreads))
    assert rc == 0, rc
    return ev


# the bytes of a warp-context record every lane of a warp shares (sm_id .. size); addr is per lane
WARP_UNIFORM = np.array([False] * 8 + [True] * 24)


def latency_pairs(n_pairs: int, seed: int = BASE_SEED, mu: float = float(np.log(20000.0)), sigma: float = 1.0,
                  n_kernels: int = 4096, out=None, nthreads=None) -> np.ndarray:
    """2*n_pairs records: (entry kind 0, exit kind 1) per block; addr low 32 bits = kernel id;
    exit.ts - entry.ts ~ round(lognormal(mu, sigma)) ns."""
    ev = _alloc(2 * n_pairs, out)
    rc = lib().evgen_latency_pairs(seed, n_pairs, mu, sigma, n_kernels, ev.ctypes.data, _threads(nthreads))
    assert rc == 0, rc
    return ev


def draw(seed: int, i: int, k: int) -> int:
    return int(lib().evgen_draw(seed, i, k))
