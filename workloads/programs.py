"""The eBPF programs the workloads run, written with the assembler in `asm.py`.

Each builder returns (slots, map_specs, ctx_size).  A map spec is a dict
{type, key_size, value_size, max_entries}.  These are inputs shared by the oracle
tests and the engine tests; they carry no execution semantics.

* counting   -- the device observability counter of the paper's `threadhist`-style tools
                (Sec. 6.4 "Low-overhead GPU Observability"): event.kind -> array-map counter.
* page_heat  -- a device memory-access policy hook (Sec. 4.3.1, `gdev_mem_ops.access`)
                keeping per-2 MiB-region heat (count, last timestamp) in a hash map, with
                an 8-iteration bounded loop and a per-kind tally.
* latency    -- a `kernelretsnoop`-style tool (Sec. 6.4): block exit - entry latency,
                log2 histogram per kernel id, outliers emitted to a ring buffer.
* warp_heat  -- page_heat's policy as a warp-level handler (Sec. 4.4.1-4.4.2) over
                warp-context records: lane addresses reach the maps only through warp
                reductions; for SIMT-aware verification and the oracle's warp run.
* sched_policy -- `should_try_steal` block-scheduling policies (FixedWork, Greedy,
                LatencyBudget) over the block context a persistent worker sees.
* random_program -- seed-generated verifier-friendly programs for the multi-program batch.
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np

from .asm import BPF_NOEXIST, MAP_ARRAY, MAP_HASH, MAP_RINGBUF, Asm

MapSpec = Dict[str, int]

# record field offsets (bytes) in the 32-byte event
F_ADDR, F_SM, F_WARP, F_TS, F_KIND, F_SIZE = 0, 8, 12, 16, 24, 28


def array_spec(n: int, value_size: int = 8) -> MapSpec:
    return dict(type=MAP_ARRAY, key_size=4, value_size=value_size, max_entries=n)


MAP_F_NO_DELETE = 1  # keys are never removed (the engine's insert-only hash maps)


def hash_spec(n: int, key_size: int = 8, value_size: int = 16, insert_only: bool = False) -> MapSpec:
    s = dict(type=MAP_HASH, key_size=key_size, value_size=value_size, max_entries=n)
    if insert_only:
        s["flags"] = MAP_F_NO_DELETE
    return s


def ringbuf_spec(nbytes: int) -> MapSpec:
    return dict(type=MAP_RINGBUF, key_size=0, value_size=0, max_entries=nbytes)


# --------------------------------------------------------------------------------------
def counting(n_counters: int = 256) -> Tuple[np.ndarray, List[MapSpec], int]:
    """key = event.kind (bounds-checked against the map size), counter += 1; returns kind."""
    a = Asm()
    a.mov("r6", "r1")
    a.ldx(4, "r7", "r6", F_KIND)
    a.ldx(4, "r3", "r6", F_SIZE)
    a.jeq("r3", 0, "out")
    a.jgt("r7", n_counters - 1, "out")
    a.stx(4, "r10", -4, "r7")
    a.ld_map("r1", 0)
    a.mov("r2", "r10")
    a.add("r2", -4)
    a.call("map_lookup_elem")
    a.jeq("r0", 0, "out")
    a.mov("r1", 1)
    a.atomic(8, "add", "r0", 0, "r1")
    a.label("out")
    a.mov("r0", "r7")
    a.exit()
    return a.prog(), [array_spec(n_counters)], 32


# --------------------------------------------------------------------------------------
PAGE_HEAT_TALLY = 16  # tally rows: 0..7 kinds, 8 = rejected record, 9 = misaligned access


def page_heat(max_entries: int = 1 << 20) -> Tuple[np.ndarray, List[MapSpec], int]:
    """Per-2 MiB-region heat.

    weight w = 1 + popcount of the 8 address bits above the 4 KiB page offset, counted by
    an 8-trip loop; region = addr >> 21; heat[region] = {count += w, last_ts = max(ts)};
    tally[kind] = {events += 1, bytes += size}; tally[9] counts size-misaligned
    addresses; records with an invalid size or kind go to tally[8] and stop.
    Maps: 0 = hash(u64 -> {u64 count, u64 last_ts}), 1 = array[16] of {u64, u64}.
    """
    a = Asm()
    a.mov("r6", "r1")
    a.ldx(8, "r7", "r6", F_ADDR)
    a.ldx(8, "r8", "r6", F_TS)
    a.ldx(4, "r2", "r6", F_SIZE)
    a.ldx(4, "r3", "r6", F_KIND)
    # size must be a power of two in [1, 4096]
    a.jeq("r2", 0, "bad")
    a.jgt("r2", 4096, "bad")
    a.mov("r4", "r2")
    a.add("r4", -1)
    a.alu("and", "r4", "r2")
    a.jne("r4", 0, "bad")
    # kind must be below 8
    a.jgt("r3", 7, "bad")
    # misaligned access -> tally[9] (and keep going)
    a.mov("r4", "r2")
    a.add("r4", -1)
    a.alu("and", "r4", "r7")
    a.jeq("r4", 0, "aligned")
    a.st(4, "r10", -28, 9)
    a.ld_map("r1", 1)
    a.mov("r2", "r10")
    a.add("r2", -28)
    a.call("map_lookup_elem")
    a.jeq("r0", 0, "aligned")
    a.mov("r1", 1)
    a.atomic(8, "add", "r0", 0, "r1")
    a.label("aligned")
    # weight loop: w = 1 + sum of bits 12..19 of addr
    a.mov("r3", "r7")
    a.rsh("r3", 12)
    a.mov("r4", 0)
    a.mov("r9", 1)
    a.label("loop")
    a.mov("r0", "r3")
    a.alu("and", "r0", 1)
    a.add("r9", "r0")
    a.rsh("r3", 1)
    a.add("r4", 1)
    a.jlt("r4", 8, "loop")
    # region key on the stack
    a.mov("r1", "r7")
    a.rsh("r1", 21)
    a.stx(8, "r10", -8, "r1")
    a.ld_map("r1", 0)
    a.mov("r2", "r10")
    a.add("r2", -8)
    a.call("map_lookup_elem")
    a.jne("r0", 0, "have")
    # insert idiom: {0, 0} with NOEXIST, then look up again
    a.st(8, "r10", -24, 0)
    a.st(8, "r10", -16, 0)
    a.ld_map("r1", 0)
    a.mov("r2", "r10")
    a.add("r2", -8)
    a.mov("r3", "r10")
    a.add("r3", -24)
    a.mov("r4", BPF_NOEXIST)
    a.call("map_update_elem")
    a.ld_map("r1", 0)
    a.mov("r2", "r10")
    a.add("r2", -8)
    a.call("map_lookup_elem")
    a.jeq("r0", 0, "out")
    a.label("have")
    a.atomic(8, "add", "r0", 0, "r9")
    a.mov("r1", "r0")
    a.add("r1", 8)
    a.mov("r2", "r8")
    a.call("atomic_max_u64")
    # per-kind tally
    a.ldx(4, "r3", "r6", F_KIND)
    a.stx(4, "r10", -28, "r3")
    a.ld_map("r1", 1)
    a.mov("r2", "r10")
    a.add("r2", -28)
    a.call("map_lookup_elem")
    a.jeq("r0", 0, "out")
    a.mov("r1", 1)
    a.atomic(8, "add", "r0", 0, "r1")
    a.ldx(4, "r2", "r6", F_SIZE)
    a.atomic(8, "add", "r0", 8, "r2")
    a.label("out")
    a.mov("r0", "r9")
    a.exit()
    a.label("bad")
    a.st(4, "r10", -28, 8)
    a.ld_map("r1", 1)
    a.mov("r2", "r10")
    a.add("r2", -28)
    a.call("map_lookup_elem")
    a.jeq("r0", 0, "bad_out")
    a.mov("r1", 1)
    a.atomic(8, "add", "r0", 0, "r1")
    a.label("bad_out")
    a.mov("r0", 0)
    a.exit()
    return a.prog(), [hash_spec(max_entries, 8, 16, insert_only=True), array_spec(PAGE_HEAT_TALLY, 16)], 32


def warp_heat(max_entries: int = 1 << 16) -> Tuple[np.ndarray, List[MapSpec], int]:
    """A warp-level memory-access policy (Sec. 4.4.1, Sec. 4.4.2) over warp-context records
    (`gen.warp_access_events`): one handler per warp, lanes in lockstep, side effects once.

    size and kind are warp-uniform and validated as in `page_heat` (a bad warp counts once in
    tally[8] and returns 0).  Lane-varying addresses reach shared state only through warp
    reductions: lo / hi = the lowest / highest 2 MiB region any lane touches, n_in = the lanes
    in region lo, n_mis = the lanes whose address is not size-aligned.  Then heat[lo] =
    {count += n_in, last_ts = max(ts)}, tally[kind] = {warps += 1, bytes += sum of sizes},
    tally[9] += n_mis, and R0 = hi - lo (the warp's region spread) in every lane.
    Maps: 0 = hash(u64 -> {u64 count, u64 last_ts}), 1 = array[16] of {u64, u64}.
    Accepted by SIMT-aware verification with the warp-uniform bytes `gen.WARP_UNIFORM`; the
    per-lane engine refuses its warp helpers.
    """
    a = Asm()
    a.mov("r6", "r1")
    a.ldx(8, "r7", "r6", F_ADDR)
    a.ldx(8, "r8", "r6", F_TS)
    a.ldx(4, "r2", "r6", F_SIZE)
    a.ldx(4, "r3", "r6", F_KIND)
    a.jeq("r2", 0, "bad")
    a.jgt("r2", 4096, "bad")
    a.mov("r4", "r2")
    a.add("r4", -1)
    a.alu("and", "r4", "r2")
    a.jne("r4", 0, "bad")
    a.jgt("r3", 7, "bad")
    # n_mis: lanes whose address is not size-aligned
    a.mov("r1", "r2")
    a.add("r1", -1)
    a.alu("and", "r1", "r7")
    a.call("warp_count")
    a.mov("r9", "r0")
    # lo, hi: the warp's lowest and highest 2 MiB region
    a.rsh("r7", 21)
    a.mov("r1", "r7")
    a.call("warp_min_u64")
    a.stx(8, "r10", -8, "r0")
    a.mov("r1", "r7")
    a.call("warp_max_u64")
    a.stx(8, "r10", -32, "r0")
    # n_in = lanes - lanes outside region lo
    a.mov("r1", "r7")
    a.ldx(8, "r2", "r10", -8)
    a.alu("sub", "r1", "r2")
    a.call("warp_count")
    a.mov("r7", "r0")
    a.mov("r1", 1)
    a.call("warp_count")
    a.alu("sub", "r0", "r7")
    a.mov("r7", "r0")
    # heat[lo]: the insert idiom, then the updates
    a.ld_map("r1", 0)
    a.mov("r2", "r10")
    a.add("r2", -8)
    a.call("map_lookup_elem")
    a.jne("r0", 0, "have")
    a.st(8, "r10", -24, 0)
    a.st(8, "r10", -16, 0)
    a.ld_map("r1", 0)
    a.mov("r2", "r10")
    a.add("r2", -8)
    a.mov("r3", "r10")
    a.add("r3", -24)
    a.mov("r4", BPF_NOEXIST)
    a.call("map_update_elem")
    a.ld_map("r1", 0)
    a.mov("r2", "r10")
    a.add("r2", -8)
    a.call("map_lookup_elem")
    a.jeq("r0", 0, "tally")
    a.label("have")
    a.atomic(8, "add", "r0", 0, "r7")
    a.mov("r1", "r0")
    a.add("r1", 8)
    a.mov("r2", "r8")
    a.call("atomic_max_u64")
    # tally[kind] += {1, sum of sizes}
    a.label("tally")
    a.ldx(4, "r1", "r6", F_SIZE)
    a.call("warp_sum_u64")
    a.mov("r7", "r0")
    a.ldx(4, "r3", "r6", F_KIND)
    a.stx(4, "r10", -36, "r3")
    a.ld_map("r1", 1)
    a.mov("r2", "r10")
    a.add("r2", -36)
    a.call("map_lookup_elem")
    a.jeq("r0", 0, "mis")
    a.mov("r1", 1)
    a.atomic(8, "add", "r0", 0, "r1")
    a.atomic(8, "add", "r0", 8, "r7")
    # tally[9] += n_mis
    a.label("mis")
    a.jeq("r9", 0, "out")
    a.st(4, "r10", -36, 9)
    a.ld_map("r1", 1)
    a.mov("r2", "r10")
    a.add("r2", -36)
    a.call("map_lookup_elem")
    a.jeq("r0", 0, "out")
    a.atomic(8, "add", "r0", 0, "r9")
    a.label("out")
    a.ldx(8, "r0", "r10", -32)
    a.ldx(8, "r1", "r10", -8)
    a.alu("sub", "r0", "r1")
    a.exit()
    a.label("bad")
    a.st(4, "r10", -36, 8)
    a.ld_map("r1", 1)
    a.mov("r2", "r10")
    a.add("r2", -36)
    a.call("map_lookup_elem")
    a.jeq("r0", 0, "bad_out")
    a.mov("r1", 1)
    a.atomic(8, "add", "r0", 0, "r1")
    a.label("bad_out")
    a.mov("r0", 0)
    a.exit()
    return a.prog(), [hash_spec(max_entries, 8, 16, insert_only=True), array_spec(PAGE_HEAT_TALLY, 16)], 32


# --------------------------------------------------------------------------------------
# Block-scheduling hook context (the `should_try_steal` hook of Sec. 4.3.2): what a worker
# block of the persistent kernel knows when its own share of work units is done and it may
# take more from the shared pool.  32 bytes, every field the same for the block's threads.
SCHED_BLOCK, SCHED_SM, SCHED_DONE, SCHED_LEFT, SCHED_ELAPSED, SCHED_BUDGET = 0, 4, 8, 12, 16, 24
SCHED_CTX = 32
SCHED_STATS = 8  # array map: per policy decision kind, {decisions, steals}


def _sched_tally(a: Asm) -> None:
    """stats[SCHED_SM & 7] = {decisions += 1, steals += r0}; r0 kept"""
    a.mov("r7", "r0")
    a.ldx(4, "r2", "r6", SCHED_SM)
    a.alu("and", "r2", 7)
    a.stx(4, "r10", -4, "r2")
    a.ld_map("r1", 0)
    a.mov("r2", "r10")
    a.add("r2", -4)
    a.call("map_lookup_elem")
    a.jeq("r0", 0, "out")
    a.mov("r1", 1)
    a.atomic(8, "add", "r0", 0, "r1")
    a.atomic(8, "add", "r0", 8, "r7")
    a.label("out")
    a.mov("r0", "r7")
    a.exit()


def sched_policy(kind: str) -> Tuple[np.ndarray, List[MapSpec], int]:
    """A `should_try_steal` policy (Sec. 4.3.2, the schedulers of Sec. 6): R0 = 1 to take
    another unit from the shared pool, 0 to stop.  FixedWork never steals; Greedy steals
    while the pool has units; LatencyBudget steals while the pool has units and the block's
    elapsed time is under its budget.  Each also counts its decisions and steals per SM
    group (array map 0, SCHED_STATS entries of {u64, u64})."""
    a = Asm()
    a.mov("r6", "r1")
    a.mov("r0", 0)
    if kind != "fixed":
        a.ldx(4, "r2", "r6", SCHED_LEFT)
        a.jeq("r2", 0, "decide")
        if kind == "latency_budget":
            a.ldx(8, "r3", "r6", SCHED_ELAPSED)
            a.ldx(8, "r4", "r6", SCHED_BUDGET)
            a.jge("r3", "r4", "decide")
        elif kind != "greedy":
            raise ValueError(kind)
        a.mov("r0", 1)
    a.label("decide")
    _sched_tally(a)
    return a.prog(), [array_spec(SCHED_STATS, 16)], SCHED_CTX


# --------------------------------------------------------------------------------------
LAT_BUCKETS = 64
OUTLIER_BYTES = 48


def lognormal_quantile_ns(mu: float, sigma: float, q: float = 0.99) -> int:
    """exp(mu + sigma * z_q), rounded; z_q from the inverse normal CDF (bisection on erf)."""
    lo, hi = -10.0, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if 0.5 * (1.0 + math.erf(mid / math.sqrt(2.0))) < q:
            lo = mid
        else:
            hi = mid
    return int(round(math.exp(mu + sigma * 0.5 * (lo + hi))))


def latency(n_kernels: int = 4096, threshold_ns: int | None = None,
            ring_bytes: int = 128 << 20) -> Tuple[np.ndarray, List[MapSpec], int]:
    """ctx = one (entry, exit) record pair (64 bytes).

    lat = exit.ts - entry.ts; bucket = floor(log2(lat)) (0 for lat = 0) by a six-step
    branchy binary search; hist[kernel_id*64 + bucket] += 1; if lat > threshold a 48-byte
    record {addr, kernel_id, bucket, entry_ts, exit_ts, lat, sm_id, warp_id} goes to the
    ring buffer.  Maps: 0 = array[n_kernels*64] of u64, 1 = ringbuf.
    """
    if threshold_ns is None:
        threshold_ns = lognormal_quantile_ns(math.log(20000.0), 1.0, 0.99)
    assert 0 < threshold_ns < 2**31
    a = Asm()
    a.mov("r6", "r1")
    a.ldx(4, "r2", "r6", F_KIND)
    a.jne("r2", 0, "out")
    a.ldx(4, "r2", "r6", 32 + F_KIND)
    a.jne("r2", 1, "out")
    a.ldx(4, "r7", "r6", F_ADDR)
    a.ldx(4, "r2", "r6", 32 + F_ADDR)
    a.jne("r2", "r7", "out")
    a.jgt("r7", n_kernels - 1, "out")
    a.ldx(8, "r8", "r6", 32 + F_TS)
    a.ldx(8, "r2", "r6", F_TS)
    a.jlt("r8", "r2", "out")
    a.sub("r8", "r2")
    # floor(log2(lat)) by halving steps
    a.mov("r9", 0)
    a.mov("r3", "r8")
    for step in (32, 16, 8, 4, 2, 1):
        a.mov("r4", "r3")
        a.rsh("r4", step)
        a.jeq("r4", 0, f"s{step}")
        a.mov("r3", "r4")
        a.add("r9", step)
        a.label(f"s{step}")
    a.mov("r2", "r7")
    a.lsh("r2", 6)
    a.add("r2", "r9")
    a.stx(4, "r10", -4, "r2")
    a.ld_map("r1", 0)
    a.mov("r2", "r10")
    a.add("r2", -4)
    a.call("map_lookup_elem")
    a.jeq("r0", 0, "out")
    a.mov("r1", 1)
    a.atomic(8, "add", "r0", 0, "r1")
    a.jle("r8", threshold_ns, "out")
    a.ld_map("r1", 1)
    a.mov("r2", OUTLIER_BYTES)
    a.mov("r3", 0)
    a.call("ringbuf_reserve")
    a.jeq("r0", 0, "out")
    a.ldx(8, "r1", "r6", F_ADDR)
    a.stx(8, "r0", 0, "r1")
    a.stx(4, "r0", 8, "r7")
    a.stx(4, "r0", 12, "r9")
    a.ldx(8, "r1", "r6", F_TS)
    a.stx(8, "r0", 16, "r1")
    a.ldx(8, "r1", "r6", 32 + F_TS)
    a.stx(8, "r0", 24, "r1")
    a.stx(8, "r0", 32, "r8")
    a.ldx(4, "r1", "r6", F_SM)
    a.stx(4, "r0", 40, "r1")
    a.ldx(4, "r1", "r6", F_WARP)
    a.stx(4, "r0", 44, "r1")
    a.mov("r1", "r0")
    a.mov("r2", 0)
    a.call("ringbuf_submit")
    a.label("out")
    a.mov("r0", 0)
    a.exit()
    return a.prog(), [array_spec(n_kernels * LAT_BUCKETS), ringbuf_spec(ring_bytes)], 64


# --------------------------------------------------------------------------------------
RANDOM_ARRAY_ENTRIES = 1024
RANDOM_HASH_ENTRIES = 4096


class _Rng:
    """SplitMix64 stream (Steele, Lea, Flood 2014) for program generation."""

    def __init__(self, seed: int) -> None:
        self.s = seed & (2**64 - 1)

    def next(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & (2**64 - 1)
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & (2**64 - 1)
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & (2**64 - 1)
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        return self.next() % n

    def choice(self, seq):
        return seq[self.below(len(seq))]


_SCALARS = ["r0", "r1", "r2", "r3", "r4", "r5", "r7", "r8", "r9"]
_ALU_BIN = ["add", "sub", "mul", "or", "and", "xor", "lsh", "rsh", "arsh", "mov", "div", "mod"]
_CMP = ["jeq", "jne", "jgt", "jge", "jlt", "jle", "jsgt", "jsge", "jslt", "jsle", "jset"]


def random_program(seed: int, target_len: int, use_hash: bool = True) -> Tuple[np.ndarray, List[MapSpec], int]:
    """A seed-generated program of about `target_len` slots that the verifier accepts.

    ALU64/ALU32 arithmetic on ctx-derived scalars, forward conditional jumps over short
    arithmetic runs, in-bounds stack spills and reloads, array-map atomics and
    hash-map insert-then-add; returns one of the scalars in r0.
    Maps: 0 = array[1024] of u64, 1 = hash(u64 -> {u64, u64}) of 4096 entries.
    """
    rng = _Rng(seed)
    a = Asm()
    lbl = [0]
    # one update operation per map keeps every result independent of event order:
    # add, or, xor and max each commute with themselves but not with one another
    arr_op = rng.choice(["add", "or", "xor", "max"])

    def fresh() -> str:
        lbl[0] += 1
        return f"L{lbl[0]}"

    a.mov("r6", "r1")
    fields = [(8, F_ADDR), (4, F_SM), (4, F_WARP), (8, F_TS), (4, F_KIND), (4, F_SIZE)]
    for r in ("r7", "r8", "r9", "r0", "r1", "r2", "r3", "r4", "r5"):
        sz, off = rng.choice(fields)
        a.ldx(sz, r, "r6", off)
    init = set(_SCALARS)
    stack_written: List[int] = []

    def alu_insn(regs) -> None:
        dst = rng.choice(regs)
        bits = 32 if rng.below(3) == 0 else 64
        op = rng.choice(_ALU_BIN + ["neg", "end"])
        if op == "neg":
            a.neg(dst, bits=bits)
        elif op == "end":
            width = rng.choice([16, 32, 64])
            order = rng.choice(["le", "be", "swap"])
            a.end(dst, width, order)
        elif op in ("lsh", "rsh", "arsh"):
            if rng.below(2) == 0:
                a.alu(op, dst, rng.below(bits), bits=bits)  # constant shifts stay below the width
            else:
                a.alu(op, dst, rng.choice(regs), bits=bits)
        elif rng.below(2) == 0:
            imm = rng.choice([1, 3, 7, 255, -1, 0x7FFF, -12345, 1 << 20, rng.below(1 << 31)])
            if op in ("div", "mod") and rng.below(4) == 0:
                a.alu(op, dst, imm, bits=bits, off=1)  # signed forms
            else:
                a.alu(op, dst, imm, bits=bits)
        else:
            a.alu(op, dst, rng.choice(regs), bits=bits)

    while len(a) < target_len - 3:
        kind = rng.below(10)
        regs = sorted(init)
        if target_len - 3 - len(a) < 32:  # near the end: single instructions only, never overshoot
            alu_insn(regs)
            continue
        if kind <= 3:
            for _ in range(1 + rng.below(5)):
                alu_insn(regs)
        elif kind == 4:
            end = fresh()
            op = rng.choice(_CMP)
            lhs = rng.choice(regs)
            if rng.below(2) == 0:
                a.jcond(op, lhs, rng.choice(regs), end, bits=rng.choice([32, 64]))
            else:
                a.jcond(op, lhs, rng.choice([0, 1, 8, 255, -1, 1000]), end, bits=rng.choice([32, 64]))
            for _ in range(1 + rng.below(4)):
                alu_insn(regs)
            a.label(end)
        elif kind == 5:
            off = -8 * (1 + rng.below(24))
            a.stx(8, "r10", off, rng.choice(regs))
            stack_written.append(off)
        elif kind == 6 and stack_written:
            off = rng.choice(stack_written)
            a.ldx(8, rng.choice(regs), "r10", off)
        elif kind == 7:
            sz, off = rng.choice(fields)
            a.ldx(sz, rng.choice(regs), "r6", off)
        elif kind == 8:
            # array map: key = reg & 1023 ; value op
            src = rng.choice([r for r in regs if r not in ("r1", "r2", "r3", "r4", "r5", "r0")] or ["r7"])
            a.mov("r2", src)
            a.alu("and", "r2", RANDOM_ARRAY_ENTRIES - 1)
            a.stx(4, "r10", -204, "r2")
            a.ld_map("r1", 0)
            a.mov("r2", "r10")
            a.add("r2", -204)
            a.call("map_lookup_elem")
            end = fresh()
            a.jeq("r0", 0, end)
            val = rng.choice(["r7", "r8", "r9"])
            op = arr_op
            if op == "max":
                a.mov("r1", "r0")
                a.mov("r2", val)
                a.call("atomic_max_u64")
            else:
                a.atomic(8, op, "r0", 0, val)
            a.label(end)
            a.mov("r0", rng.below(1000))
            init -= {"r1", "r2", "r3", "r4", "r5"}
            for r in ("r1", "r2", "r3", "r4", "r5"):
                if rng.below(2) == 0:
                    a.mov(r, rng.below(1 << 16))
                    init.add(r)
        elif kind == 9 and use_hash:
            src = rng.choice(["r7", "r8", "r9"])
            a.mov("r2", src)
            a.alu("and", "r2", 0xFFF)
            a.stx(8, "r10", -216, "r2")
            have, end = fresh(), fresh()
            a.ld_map("r1", 1)
            a.mov("r2", "r10")
            a.add("r2", -216)
            a.call("map_lookup_elem")
            a.jne("r0", 0, have)
            a.st(8, "r10", -232, 0)
            a.st(8, "r10", -224, 0)
            a.ld_map("r1", 1)
            a.mov("r2", "r10")
            a.add("r2", -216)
            a.mov("r3", "r10")
            a.add("r3", -232)
            a.mov("r4", BPF_NOEXIST)
            a.call("map_update_elem")
            a.ld_map("r1", 1)
            a.mov("r2", "r10")
            a.add("r2", -216)
            a.call("map_lookup_elem")
            a.jeq("r0", 0, end)
            a.label(have)
            a.atomic(8, "add", "r0", 0, rng.choice(["r7", "r8", "r9"]))
            a.mov("r1", "r0")
            a.add("r1", 8)
            a.mov("r2", rng.choice(["r7", "r8", "r9"]))
            a.call("atomic_max_u64")
            a.label(end)
            a.mov("r0", rng.below(1000))
            init -= {"r1", "r2", "r3", "r4", "r5"}
    a.mov("r0", rng.choice(sorted(init - {"r0"}) or ["r7"]))
    a.exit()
    maps = [array_spec(RANDOM_ARRAY_ENTRIES), hash_spec(RANDOM_HASH_ENTRIES, 8, 16, insert_only=True)]
    return a.prog(), maps, 32


def batch_programs(n_programs: int = 64, seed: int = 0x6758, min_len: int = 10, max_len: int = 400):
    """The multi-program workload: program p has length uniform in [min_len, max_len]."""
    rng = _Rng(seed ^ 0xB47C4)
    out = []
    for p in range(n_programs):
        length = min_len + rng.below(max_len - min_len + 1)
        out.append(random_program(seed ^ (p * 0x9E3779B1), length))
    return out


def batch_sizes(n_programs: int = 64, seed: int = 0x6758, lo: int = 4096, hi: int = 16 << 20) -> List[int]:
    """Event-batch sizes, log-uniform over [lo, hi]."""
    rng = _Rng(seed ^ 0x51235)
    out = []
    for _ in range(n_programs):
        u = (rng.next() >> 11) / float(1 << 53)
        out.append(int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))))
    return out
