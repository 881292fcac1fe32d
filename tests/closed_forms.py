"""Closed forms of what the workload programs compute, written directly with numpy.

They restate each program's intent on the event arrays (no eBPF involved), so they pin
both the oracle and, at sizes the oracle cannot reach quickly, the engine:
  counting  -> bincount of event.kind
  page_heat -> group-by of addr >> 21: (sum of weights, max timestamp); per-kind tally
  latency   -> 2-D histogram of (kernel id, floor(log2(latency))); outliers latency > T
  warp_heat -> per warp: lowest / highest region, lanes in the lowest, sizes, misaligned lanes
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

from workloads import programs as P


def counting(ev: np.ndarray, n_counters: int = 256) -> np.ndarray:
    k = ev["kind"].astype(np.int64)
    ok = (ev["size"] != 0) & (k < n_counters)
    return np.bincount(k[ok], minlength=n_counters).astype(np.uint64)


def popcount8(x: np.ndarray) -> np.ndarray:
    x = x & 0xFF
    c = np.zeros_like(x)
    for b in range(8):
        c += (x >> b) & 1
    return c


def page_heat(ev: np.ndarray) -> Tuple[Dict[int, Tuple[int, int]], np.ndarray]:
    """({region: (count, last_ts)}, tally[16, 2]) for records the program accepts."""
    addr, size, kind, ts = ev["addr"], ev["size"].astype(np.uint64), ev["kind"].astype(np.uint64), ev["ts_ns"]
    pow2 = (size != 0) & (size <= 4096) & ((size & (size - np.uint64(1))) == 0)
    ok = pow2 & (kind < 8)
    tally = np.zeros((P.PAGE_HEAT_TALLY, 2), dtype=np.uint64)
    tally[8, 0] = np.count_nonzero(~ok)
    a, s, k, t = addr[ok], size[ok], kind[ok], ts[ok]
    mis = (a & (s - np.uint64(1))) != 0
    tally[9, 0] = np.count_nonzero(mis)
    tally[:8, 0] = np.bincount(k.astype(np.int64), minlength=8)[:8]
    tally[:8, 1] = np.bincount(k.astype(np.int64), weights=s.astype(np.float64), minlength=8)[:8].astype(np.uint64)
    w = np.uint64(1) + popcount8(a >> np.uint64(12))
    region = a >> np.uint64(21)
    order = np.argsort(region, kind="stable")
    r_sorted = region[order]
    uniq, starts = np.unique(r_sorted, return_index=True)
    sums = np.add.reduceat(w[order], starts)
    maxts = np.maximum.reduceat(t[order], starts)
    heat = {int(u): (int(c), int(m)) for u, c, m in zip(uniq, sums, maxts)}
    return heat, tally


def floor_log2(x: np.ndarray) -> np.ndarray:
    """floor(log2(x)) per element, 0 for x = 0 (count of k in 1..63 with x >> k != 0).
    Below 2^53 every value is exact in binary64 and frexp's exponent gives the same count."""
    x = np.asarray(x, dtype=np.uint64)
    if x.size and int(x.max()) < (1 << 53):
        _, e = np.frexp(x.astype(np.float64))
        return np.maximum(e.astype(np.int64) - 1, 0)
    b = np.zeros(x.shape, dtype=np.int64)
    for k in range(1, 64):
        b += (x >> np.uint64(k)) > 0
    return b


OUTLIER_DTYPE = np.dtype([("addr", "<u8"), ("kid", "<u4"), ("bucket", "<u4"), ("ets", "<u8"), ("xts", "<u8"),
                          ("lat", "<u8"), ("sm", "<u4"), ("warp", "<u4")])


def latency(ev: np.ndarray, n_kernels: int = 4096, threshold: int | None = None):
    """(hist[n_kernels*64] u64, outliers [(pair index, payload bytes)] in index order)."""
    if threshold is None:
        import math
        threshold = P.lognormal_quantile_ns(math.log(20000.0), 1.0, 0.99)
    e, x = ev[0::2], ev[1::2]
    kid = (e["addr"] & np.uint64(0xFFFFFFFF))
    ok = (e["kind"] == 0) & (x["kind"] == 1) & ((x["addr"] & np.uint64(0xFFFFFFFF)) == kid)
    ok &= kid < n_kernels
    ok &= x["ts_ns"] >= e["ts_ns"]
    lat = (x["ts_ns"] - e["ts_ns"])
    b = floor_log2(lat)
    idx = kid[ok].astype(np.int64) * P.LAT_BUCKETS + b[ok]
    hist = np.bincount(idx, minlength=n_kernels * P.LAT_BUCKETS).astype(np.uint64)
    sel, recs = latency_outliers(e, x, kid, b, lat, ok, threshold)
    out: List[Tuple[int, bytes]] = [(int(i), recs[k].tobytes()) for k, i in enumerate(sel)]
    return hist, out


def latency_outliers(e, x, kid, b, lat, ok, threshold):
    """(pair indices in order, OUTLIER_DTYPE payloads) of the pairs with latency > threshold."""
    sel = np.nonzero(ok & (lat > np.uint64(threshold)))[0]
    recs = np.zeros(len(sel), dtype=OUTLIER_DTYPE)
    recs["addr"], recs["kid"], recs["bucket"] = e["addr"][sel], kid[sel], b[sel]
    recs["ets"], recs["xts"], recs["lat"] = e["ts_ns"][sel], x["ts_ns"][sel], lat[sel]
    recs["sm"], recs["warp"] = e["sm_id"][sel], e["warp_id"][sel]
    return sel, recs


def latency_arrays(ev: np.ndarray, n_kernels: int = 4096, threshold: int | None = None):
    """latency() for large batches: (hist, outlier pair indices, OUTLIER_DTYPE payloads)."""
    if threshold is None:
        import math
        threshold = P.lognormal_quantile_ns(math.log(20000.0), 1.0, 0.99)
    e, x = ev[0::2], ev[1::2]
    kid = (e["addr"] & np.uint64(0xFFFFFFFF))
    ok = (e["kind"] == 0) & (x["kind"] == 1) & ((x["addr"] & np.uint64(0xFFFFFFFF)) == kid)
    ok &= kid < n_kernels
    ok &= x["ts_ns"] >= e["ts_ns"]
    lat = (x["ts_ns"] - e["ts_ns"])
    b = floor_log2(lat)
    idx = kid[ok].astype(np.int64) * P.LAT_BUCKETS + b[ok]
    hist = np.bincount(idx, minlength=n_kernels * P.LAT_BUCKETS).astype(np.uint64)
    sel, recs = latency_outliers(e, x, kid, b, lat, ok, threshold)
    return hist, sel, recs


def warp_heat(ev: np.ndarray, lanes: int = 32) -> Tuple[Dict[int, Tuple[int, int]], np.ndarray, np.ndarray]:
    """({region: (count, last_ts)}, tally[16, 2], R0 per record) of the warp-level policy:
    warps of `lanes` consecutive records (the last may be shorter); per warp lo / hi = the
    lowest / highest addr >> 21, heat[lo] gains the lanes in region lo and the warp's ts,
    tally[kind] one warp and the sizes, tally[9] the misaligned lanes; R0 = hi - lo."""
    heat: Dict[int, Tuple[int, int]] = {}
    tally = np.zeros((P.PAGE_HEAT_TALLY, 2), dtype=np.uint64)
    r0 = np.zeros(len(ev), dtype=np.int64)
    for w0 in range(0, len(ev), lanes):
        w = ev[w0:w0 + lanes]
        size, kind, ts = int(w["size"][0]), int(w["kind"][0]), int(w["ts_ns"][0])
        if not (0 < size <= 4096 and size & (size - 1) == 0 and kind < 8):
            tally[8, 0] += np.uint64(1)
            continue
        region = w["addr"] >> np.uint64(21)
        lo, hi = int(region.min()), int(region.max())
        count, last = heat.get(lo, (0, 0))
        heat[lo] = (count + int(np.count_nonzero(region == lo)), max(last, ts))
        tally[kind, 0] += np.uint64(1)
        tally[kind, 1] += np.uint64(size * len(w))
        tally[9, 0] += np.uint64(np.count_nonzero(w["addr"] & np.uint64(size - 1)))
        r0[w0:w0 + lanes] = hi - lo
    return heat, tally, r0
