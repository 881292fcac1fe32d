"""Merging map copies built by several engines, at read time: the multi-GPU path.

Each engine (one per GPU) runs the same program over its own part of a batch with maps of
its own.  Under deterministic verification a map's final contents do not depend on the order
of the updates, so the copies combine exactly into the map one engine would have built over
the whole batch (Sec. 5.3: GPU-local shards merged into a canonical snapshot at
synchronisation points).  `gx_merge_ops` says how each 4-byte word of a value combines; the
functions here apply it to host snapshots (`Map.array_values`, `Map.hash_items`, a drained
ring's records) and `allgather_merge` does it across torch.distributed ranks.
"""
from __future__ import annotations

from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import gx as G

_REDUCE = {G.MERGE_OR: np.bitwise_or, G.MERGE_AND: np.bitwise_and, G.MERGE_MAX: np.maximum, G.MERGE_MIN: np.minimum}


def groups(word_ops: Sequence[int], value_size: int) -> List[Tuple[int, int, int]]:
    """(byte offset, width, op) for each update group of a value; a 64-bit update spans two
    words.  Bytes no update reaches form (offset, width, MERGE_NONE) groups."""
    out, w = [], 0
    while w < len(word_ops):
        c = int(word_ops[w])
        if c & G.MERGE_W8:
            out.append((4 * w, 8, c & 0xF))
            w += 2
        else:
            out.append((4 * w, min(4, value_size - 4 * w), c))
            w += 1
    return out


def _column(raw: np.ndarray, off: int, width: int) -> np.ndarray:
    """bytes [off, off + width) of each row as one little-endian uint64"""
    col = np.zeros(raw.shape[0], dtype=np.uint64)
    for b in range(width):
        col |= raw[:, off + b].astype(np.uint64) << np.uint64(8 * b)
    return col


def _store(raw: np.ndarray, off: int, width: int, col: np.ndarray) -> None:
    for b in range(width):
        raw[:, off + b] = ((col >> np.uint64(8 * b)) & np.uint64(0xFF)).astype(np.uint8)


def _merge_rows(vals: np.ndarray, who: np.ndarray, n_out: int, start: np.ndarray,
                word_ops: Sequence[int]) -> np.ndarray:
    """Merge value rows `vals` (uint8, rows x value_size) into `n_out` rows: row r belongs to
    output who[r]; start (n_out x value_size) holds each output's starting value."""
    value_size = vals.shape[1]
    out = start.copy()
    for off, width, op in groups(word_ops, value_size):
        mask = np.uint64((1 << (8 * width)) - 1)
        v, i = _column(vals, off, width), _column(start, off, width)
        if op == G.MERGE_NONE:  # no update changes these bytes: every copy holds the same, take the first
            first = np.full(n_out, len(who), dtype=np.int64)
            np.minimum.at(first, who, np.arange(len(who)))
            has = first < len(who)
            acc = i.copy()
            acc[has] = v[first[has]]
            if np.any(v != acc[who]):
                raise ValueError(f"bytes [{off}, {off + width}) differ between copies but no update changes them")
        elif op == G.MERGE_ADD:
            acc = i.copy()
            np.add.at(acc, who, (v - i[who]) & mask)
        elif op == G.MERGE_XOR:
            acc = i.copy()
            np.bitwise_xor.at(acc, who, v ^ i[who])
        elif op in _REDUCE:
            acc = i.copy()
            _REDUCE[op].at(acc, who, v)
        else:
            raise ValueError(f"unknown merge code {op}")
        _store(out, off, width, acc & mask)
    return out


def merge_array(word_ops: Sequence[int], copies: Sequence[np.ndarray], init: Optional[np.ndarray] = None) -> np.ndarray:
    """Merge array-map copies (each max_entries x value_size bytes, as `Map.array_values`).
    init: the contents every copy started from (zeros by default)."""
    shape = np.asarray(copies[0]).shape
    start = np.zeros(shape, dtype=np.uint8) if init is None else np.asarray(init, dtype=np.uint8).reshape(shape)
    vals = np.concatenate([np.asarray(c, dtype=np.uint8).reshape(shape) for c in copies])
    who = np.tile(np.arange(shape[0]), len(copies))
    return _merge_rows(vals, who, shape[0], start, word_ops)


def merge_hash(word_ops: Sequence[int], copies: Sequence[Dict[bytes, bytes]], insert: Optional[bytes] = None,
               init: Optional[Dict[bytes, bytes]] = None) -> Dict[bytes, bytes]:
    """Merge hash-map copies ({key: value} as `Map.hash_items`): the union of the keys, each
    merged over the copies that hold it.  A key starts from init[key] when the map held it
    before the runs, else from the program's insert constant `insert`."""
    keys = sorted({k for c in copies for k in c})
    if not keys:
        return {}
    pos = {k: j for j, k in enumerate(keys)}
    value_size = len(next(iter(next(c for c in copies if c).values())))
    rows, who = [], []
    for c in copies:
        for k, v in c.items():
            rows.append(np.frombuffer(v, dtype=np.uint8))
            who.append(pos[k])
    start = np.zeros((len(keys), value_size), dtype=np.uint8)
    for j, k in enumerate(keys):
        if init is not None and k in init:
            start[j] = np.frombuffer(init[k], dtype=np.uint8)
        elif insert is not None:
            start[j] = np.frombuffer(insert, dtype=np.uint8)
        elif sum(k in c for c in copies) > 1 and any(op in (G.MERGE_ADD, G.MERGE_XOR) for _, _, op in
                                                     groups(word_ops, value_size)):
            raise ValueError("a key held by several copies needs its starting value (init or insert)")
    merged = _merge_rows(np.stack(rows), np.asarray(who), len(keys), start, word_ops)
    return {k: merged[j].tobytes() for j, k in enumerate(keys)}


def merge_ring(copies: Sequence[Tuple[List[Tuple[int, bytes]], int]]) -> Tuple[List[Tuple[int, bytes]], int]:
    """Merge ring-buffer drains ((records as (event_idx, payload), dropped) per copy): the
    records of all copies ordered by event index, keeping each event's emission order, and
    the drops summed.  Event indices are global (each engine ran with its part's base)."""
    records = [r for recs, _ in copies for r in recs]
    records.sort(key=lambda r: r[0])  # stable: one event's records come from one copy, in order
    return records, sum(int(d) for _, d in copies)


def allgather_merge(dist, local, merge: Callable[[list], object]):
    """Across torch.distributed ranks: gather every rank's snapshot `local` (any picklable
    object) and return merge(list of snapshots in rank order) on every rank."""
    copies = [None] * dist.get_world_size()
    dist.all_gather_object(copies, local)
    return merge(copies)


def merge_snapshots(prog: np.ndarray, specs: Sequence[dict], ctx_size: int, copies: Sequence[Sequence],
                    init: Optional[Sequence[Optional[np.ndarray]]] = None) -> list:
    """Merge every map of one program at once.  copies[c][m] is engine c's snapshot of map m:
    array bytes (max_entries x value_size), a {key: value} dict, or a ring's (records,
    dropped).  init[m]: the contents array map m started from (None: zeros).  Raises
    ValueError when gx_merge_ops refuses the program or a map (its log says why)."""
    out = []
    for m, spec in enumerate(specs):
        parts = [c[m] for c in copies]
        if spec["type"] == G.MAP_RINGBUF:
            out.append(merge_ring(parts))
            continue
        rc, ops, insert, log = G.merge_ops(prog, specs, ctx_size, m)
        if rc != 0:
            raise ValueError(f"map {m} cannot be merged: {log}")
        if spec["type"] == G.MAP_ARRAY:
            start = None if init is None or init[m] is None else np.asarray(init[m], dtype=np.uint8)
            out.append(merge_array(ops, parts, init=start))
        else:
            out.append(merge_hash(ops, parts, insert=insert))
    return out


def merge_across_ranks(dist, prog: np.ndarray, specs: Sequence[dict], ctx_size: int, local: Sequence,
                       init: Optional[Sequence[Optional[np.ndarray]]] = None) -> list:
    """Every rank passes its own snapshots of the program's maps; every rank gets the merged
    maps (merge_snapshots over the ranks' snapshots, in rank order)."""
    return allgather_merge(dist, list(local), lambda copies: merge_snapshots(prog, specs, ctx_size, copies, init))
