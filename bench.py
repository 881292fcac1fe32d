#!/usr/bin/env python3
"""Benchmark of the device-side eBPF engine on one GB300 (or N, one process per GPU).

Headline (one JSON line on stdout): the page-heat policy (~90-slot program with an
8-trip loop, hash map of 1M entries + per-kind array tally) over 64M 32-byte events with
Zipf(1.1) page addresses over a 64 GiB space; one step = one plain launch of the
load-time specialised program over the whole batch, maps resident across steps (the
interpreter's figures are under "configs").  After the timed steps the maps are checked
against the closed form of the policy at full size ("parity"); a mismatch fails the run.
The line also carries
the roofline of that kernel, the oracle's CPU throughput on a bounded sample, the same
metric end to end through host buffers, the clocks seen during the timed region and,
under "configs", the other workloads: counting (1M events, L2 flushed between reps),
latency (256M records as 128M pairs, ring-buffer outliers), the 64-program batch
(64 plain launches vs one persistent-kernel graph launch) and the served form
(Poisson arrivals, continuous batching vs one launch per request, p50/p99).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--only headline]
Under torchrun each rank runs its own batch (weak scaling, no data-path collective);
rank 0 prints the line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import gen  # noqa: E402
from workloads import programs as P  # noqa: E402

C2_EVENTS = 64 << 20
C1_EVENTS = 1 << 20
C3_PAIRS = 128 << 20
SEED = 0x6758
# DRAM bytes (read + write) per event of the specialised page-heat kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of a 16M-event launch; traffic grows with the
# events streamed, so a launch's traffic is this figure times its events.  Re-take it whenever
# that kernel changes.
PAGEHEAT_JIT_DRAM_BYTES_PER_EVENT = (543.648768e6 + 5.825792e6) / 16777216
PAGEHEAT_WORKLOAD = ("page-heat policy, 64M events/GPU, Zipf(1.1) 4 KiB pages over 64 GiB, "
                     "hash map 1M entries (u64 -> {count, last_ts}), 8-trip loop")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 100 ms while running; summary over samples under load."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,utilization.gpu,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,clocks.mem,"
              "temperature.memory")

    def __init__(self, index: int) -> None:
        self.index = index
        self.samples = []
        self.proc = None

    def start(self) -> None:
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self) -> None:
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                self.samples.append(parts)

    def stop(self) -> dict:
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()
        busy = [s for s in self.samples if s[3].isdigit() and int(s[3]) > 20] or self.samples
        if not busy:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = sorted(float(s[1]) for s in busy if s[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in busy for k in range(4) if s[6 + k].strip() in ("Active", "1")})
        mem = sorted(float(s[10]) for s in busy if len(s) > 10 and s[10].replace(".", "").isdigit())
        temp = sorted(float(s[11]) for s in busy if len(s) > 11 and s[11].replace(".", "").isdigit())
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": float(busy[0][2]) if busy[0][2] else None,
                "reasons": reasons, "samples": len(busy), "mem_mhz": mem[len(mem) // 2] if mem else None,
                "mem_temp_c_max": temp[-1] if temp else None}


# ---------------------------------------------------------------------------- helpers
def to_device(ev: np.ndarray):
    import torch

    raw = np.ascontiguousarray(ev).view(np.uint8).reshape(-1)
    return torch.from_numpy(raw).cuda()


def flush_l2(buf) -> None:
    buf.add_(1)


class EventTimer:
    def __init__(self, stream) -> None:
        import torch

        self.s = stream
        self.a = torch.cuda.Event(enable_timing=True)
        self.b = torch.cuda.Event(enable_timing=True)

    def __enter__(self):
        self.a.record(self.s)
        return self

    def __exit__(self, *exc):
        self.b.record(self.s)

    def ms(self) -> float:
        self.b.synchronize()
        return self.a.elapsed_time(self.b)


# ---------------------------------------------------------------------------- full-size result checks
def check_pageheat(maps, ev, launches: int) -> dict:
    """The maps after `launches` launches over the whole batch against the closed form of
    page-heat (tests/closed_forms.py: group-by of addr >> 21 of (sum of weights, max ts), and
    the per-kind tally), counts scaled by the launch count.  Bit-exact."""
    from tests import closed_forms as CF

    heat, tally = CF.page_heat(ev)
    got = maps[0].hash_items()
    bad_keys = set(got) ^ {int(k).to_bytes(8, "little") for k in heat}
    bad_vals = 0
    for k, (c, t) in heat.items():
        v = got.get(int(k).to_bytes(8, "little"))
        if v is not None and (int.from_bytes(v[:8], "little") != c * launches or
                              int.from_bytes(v[8:16], "little") != t):
            bad_vals += 1
    tally_ok = bool(np.array_equal(maps[1].array_u64(), tally * np.uint64(launches)))
    ok = not bad_keys and bad_vals == 0 and tally_ok
    return {"ok": ok, "what": "hash map and tally vs closed form x launches", "launches": launches,
            "keys": len(heat), "keys_differing": len(bad_keys), "values_differing": bad_vals, "tally_ok": tally_ok}


def parse_ring_fixed(raw: bytes, payload: int):
    """Records of one payload size from a drained ring: (event indices, payload bytes rows)."""
    rec = 16 + ((payload + 7) & ~7)
    a = np.frombuffer(raw, dtype=np.uint8)
    assert a.size % rec == 0, "ring stream is not a whole number of records"
    a = a.reshape(-1, rec)
    lens = a[:, :4].copy().view("<u4")[:, 0]
    assert (lens == payload).all(), "unexpected record length"
    return a[:, 8:16].copy().view("<u8")[:, 0], a[:, 16:16 + payload]


def check_latency(maps, ev, launches: int, raw_last: bytes, dropped_last: int) -> dict:
    """The histogram after `launches` launches against the closed form (2-D histogram of
    kernel id and floor(log2(latency))) times the launch count, and the last launch's drained
    outlier records, sorted by pair index, against the closed form's outliers byte for byte."""
    from tests import closed_forms as CF

    hist, sel, recs = CF.latency_arrays(ev)
    hist_ok = bool(np.array_equal(maps[0].array_u64()[:, 0], hist * np.uint64(launches)))
    idx, pay = parse_ring_fixed(raw_last, CF.OUTLIER_DTYPE.itemsize)
    order = np.argsort(idx, kind="stable")
    ring_ok = (dropped_last == 0 and len(idx) == len(sel) and bool(np.array_equal(idx[order], sel)) and
               bool(np.array_equal(pay[order], recs.view(np.uint8).reshape(len(recs), -1))))
    return {"ok": hist_ok and ring_ok, "what": "histogram vs closed form x launches; last launch's outlier "
                                               "records vs closed form, sorted by pair index",
            "launches": launches, "hist_ok": hist_ok, "ring_ok": ring_ok, "outliers": int(len(sel))}


def oracle_insns(prog, specs, cs, ev, n_sample) -> float:
    import oracle as O

    om = O.maps_from_specs(specs)
    _, cnt = O.run(prog, om, ev[:n_sample * (cs // 32)], cs)
    return cnt / n_sample


# ---------------------------------------------------------------------------- ranks (weak scaling)
def rank_seed(rank: int) -> int:
    """Each rank streams its own batch: same recipe, its own seed (no data-path collective)."""
    return SEED ^ rank


def job_rate(torch, local_ms: float, world: int, units_per_rank: int, device=None):
    """(slowest rank's time, whole-job millions of units per second): every rank processed
    units_per_rank units, and the job took as long as its slowest rank."""
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * units_per_rank / (ms / 1e3) / 1e6


# ---------------------------------------------------------------------------- headline: page heat
def run_headline(args, gx, torch, dist_env, jit=True):
    rank, world = dist_env
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    prog_i, specs, cs = P.page_heat()
    ev = gen.pageheat_events(C2_EVENTS, seed=rank_seed(rank))
    dev = to_device(ev)
    ctx = gx.Context(torch.cuda.current_device())
    maps = [gx.Map.from_spec(ctx, s) for s in specs]
    prog = gx.Program(ctx, prog_i, maps, cs, deterministic=True, jit=jit)
    block, ept, shards = prog.autotune(dev, C2_EVENTS, stream=sid)
    variant = getattr(prog, "tuned_variant", 0)
    grid = "one wave" if getattr(prog, "tuned_grid", 0) == 0 else "one block per chunk"
    torch.cuda.synchronize()
    launches = 0  # every launch into the resident maps, for the full-size result check
    for _ in range(args.warmup):
        prog.run(dev, C2_EVENTS, stream=sid)
        launches += 1
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.25)
    # the timed region: K plain launches, each one pass over the whole 2 GiB batch (> L2)
    reps = max(1, args.steps)
    per = []
    t_all = EventTimer(stream)
    with t_all:
        for _ in range(reps):
            t = EventTimer(stream)
            with t:
                prog.run(dev, C2_EVENTS, stream=sid)
            per.append(t)
    total_ms = t_all.ms()
    launches += reps
    launch_ms = [t.ms() for t in per]
    # keep sampling clocks over a longer busy window so the summary has samples
    t_end = time.time() + 1.5
    while time.time() < t_end:
        for _ in range(20):
            prog.run(dev, C2_EVENTS, stream=sid)
            launches += 1
        torch.cuda.synchronize()
    clk = clocks.stop()
    st = prog.status()
    assert st.status == 0, f"device status {st.status}"
    parity = check_pageheat(maps, ev, launches)
    total_ms, _ = job_rate(torch, total_ms, world, C2_EVENTS * reps, device="cuda")
    ms_step = total_ms / reps
    value = world * C2_EVENTS / (ms_step / 1e3) / 1e6
    avg_launch = sum(launch_ms) / len(launch_ms)
    # the paper averages its trials by the geometric mean (Sec. 6 setup): per-step throughputs
    geomean_steps = float(np.exp(np.mean(np.log([C2_EVENTS / (ms / 1e3) / 1e6 for ms in launch_ms if ms > 0]))))
    peak, peak_kind = peaks()
    algo_bytes = C2_EVENTS * 32
    achieved = algo_bytes / (avg_launch / 1e3) / 1e9
    # end to end: host buffers through the C ABI, copies inside the timed region
    e2e = None
    if not args.skip_e2e and jit:
        pinned = torch.empty(C2_EVENTS * 32, dtype=torch.uint8).pin_memory()
        pinned.numpy()[:] = ev.view(np.uint8).reshape(-1)
        hb = pinned.numpy()
        snap_bytes = 0
        prog.run_host(hb.view(gen.EVENT_DTYPE))  # warm the staging buffers
        n_e2e = max(2, min(reps, 5))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            prog.run_host(hb.view(gen.EVENT_DTYPE))
            items = maps[0].hash_items()
            tally = maps[1].array_values()
            snap_bytes = len(items) * 24 + tally.nbytes
        e2e_s = (time.perf_counter() - t0) / n_e2e
        e2e = {"value": round(C2_EVENTS / e2e_s / 1e6, 1), "unit": "Mevents/s", "h2d_bytes_per_step": C2_EVENTS * 32,
               "d2h_bytes_per_step": snap_bytes, "ms_per_step": round(e2e_s * 1e3, 3),
               "path": "gx_run_batch_host (pinned host events, 2-stream chunked H2D) + gx_map_read of both maps"}
    insns_per_event = oracle_insns(prog_i, specs, cs, ev, 1 << 20)
    res = {
        "value": round(value, 1), "ms_per_step": round(ms_step, 4), "gpu_launches": reps,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": round(PAGEHEAT_JIT_DRAM_BYTES_PER_EVENT * C2_EVENTS) if jit else None,
                     "traffic_source": "ncu capture of 16M events scaled to the launch" if jit else None,
                     "peak_kind": peak_kind,
                     "kernel": "gx_jit_kernel" if jit else "gx_exec_kernel", "algorithmic_bytes_per_launch": algo_bytes,
                     "avg_launch_ms": round(avg_launch, 4)},
        "clocks": clk, "e2e": e2e, "launch_shape": {"block": block, "ept": ept, "shards": shards, "variant": variant, "grid": grid},
        "insns_per_event": round(insns_per_event, 2),
        "Minsns_per_s": round(value * insns_per_event, 1),
        "Mevents_per_s_geomean_steps": round(geomean_steps, 1),
        "parity": parity,
    }
    prog.destroy()
    for m in maps:
        m.destroy()
    ctx.close()
    del dev
    return res


# ---------------------------------------------------------------------------- other configs
def run_counting(gx, torch, jit=True):
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    prog_i, specs, cs = P.counting()
    ev = gen.uniform_events(C1_EVENTS, seed=SEED)
    dev = to_device(ev)
    ctx = gx.Context(torch.cuda.current_device())
    maps = [gx.Map.from_spec(ctx, s) for s in specs]
    prog = gx.Program(ctx, prog_i, maps, cs, deterministic=True, jit=jit)
    prog.autotune(dev, C1_EVENTS, stream=sid)
    flush = torch.zeros(64 << 20, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    times = []
    for r in range(13):
        flush_l2(flush)
        t = EventTimer(stream)
        with t:
            prog.run(dev, C1_EVENTS, stream=sid)
        if r >= 3:
            times.append(t.ms())
    ms = float(np.median(times))
    out = {"workload": "counting 1M events, 256 u64 counters", "Mevents_per_s": round(C1_EVENTS / ms / 1e3, 1),
           "kernel_ms_median": round(ms, 4), "GBps": round(C1_EVENTS * 32 / ms / 1e6, 1), "l2": "flushed per rep"}
    prog.destroy()
    for m in maps:
        m.destroy()
    ctx.close()
    return out


def run_latency(gx, torch, jit=True, pairs=None):
    pairs = pairs or C3_PAIRS
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    prog_i, specs, cs = P.latency()
    ev = gen.latency_pairs(pairs, seed=SEED)
    dev = to_device(ev)
    ctx = gx.Context(torch.cuda.current_device())
    maps = [gx.Map.from_spec(ctx, s) for s in specs]
    prog = gx.Program(ctx, prog_i, maps, cs, deterministic=True, jit=jit)
    tuned = prog.autotune(dev, pairs, stream=sid) + (prog.tuned_variant,)
    times = []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.25)
    for r in range(8):
        t = EventTimer(stream)
        with t:
            prog.run(dev, pairs, stream=sid)
        ms = t.ms()
        raw, dropped = maps[1].drain(stream=sid)
        if r >= 2:
            times.append(ms)
    clk = clocks.stop()
    assert prog.status().status == 0
    parity = check_latency(maps, ev, 8, raw, dropped)
    del ev
    ms = float(np.median(times))
    nbytes = pairs * 64 + len(raw)
    peak, _ = peaks()
    out = {"workload": f"latency {2 * pairs} records ({pairs} entry/exit pairs), 4096x64 histogram, 1% outliers "
                       "to ringbuf",
           "Mevents_per_s": round(2 * pairs / ms / 1e3, 1), "Mpairs_per_s": round(pairs / ms / 1e3, 1),
           "kernel_ms_median": round(ms, 4), "GBps": round(nbytes / ms / 1e6, 1),
           "hbm_frac": round(nbytes / ms / 1e6 / peak, 4), "ringbuf_bytes": len(raw), "dropped": dropped,
           "launch": {**dict(zip(("block", "ept", "shards", "variant"), tuned)),
                      "grid": "one block per chunk" if prog.tuned_grid == gx.GRID_PER_CHUNK else "one wave"},
           "clocks": clk,
           "kernel_ms_all": [round(t, 4) for t in times], "parity": parity}
    prog.destroy()
    for m in maps:
        m.destroy()
    ctx.close()
    return out


def build_batch(gx, torch, ctx, sizes, seed=SEED, jit=True):
    progs = P.batch_programs(seed=seed)
    items = []
    for p, ((prog_i, specs, cs), n) in enumerate(zip(progs, sizes)):
        maps = [gx.Map.from_spec(ctx, s) for s in specs]
        prog = gx.Program(ctx, prog_i, maps, cs, deterministic=True, jit=jit)
        ev = gen.uniform_events(n, seed=seed ^ p)
        items.append((prog, maps, to_device(ev), n))
    return items


def run_batched(gx, torch):
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    sizes = P.batch_sizes()
    ctx = gx.Context(torch.cuda.current_device())
    items = build_batch(gx, torch, ctx, sizes)
    total = sum(sizes)
    # planning tunes each program's map sharding (and the batch's launch shape) on scratch maps; the
    # plain launches below use the same per-program choices
    b = gx.Batch(ctx)
    for prog, _, dev, n in items:
        b.add(prog, dev, n)
    b.plan(stream=sid)
    # plain: 64 launches
    for _ in range(2):
        for prog, _, dev, n in items:
            prog.run(dev, n, stream=sid)
    tp = []
    for _ in range(5):
        t = EventTimer(stream)
        with t:
            for prog, _, dev, n in items:
                prog.run(dev, n, stream=sid)
        tp.append(t.ms())
    for _ in range(2):
        b.launch(stream=sid)
    tb = []
    for _ in range(5):
        t = EventTimer(stream)
        with t:
            b.launch(stream=sid)
        tb.append(t.ms())
    mp, mb = float(np.median(tp)), float(np.median(tb))
    out = {"workload": f"64 generated programs (12-391 slots) over log-uniform batches 4K-16M, {total} events",
           "plain_64_launches": {"ms": round(mp, 3), "Mevents_per_s": round(total / mp / 1e3, 1)},
           "batched_graph": {"ms": round(mb, 3), "Mevents_per_s": round(total / mb / 1e3, 1)},
           "speedup": round(mp / mb, 3)}
    b.destroy()
    for prog, maps, dev, n in items:
        prog.destroy()
        for m in maps:
            m.destroy()
    ctx.close()
    return out


def run_sched(gx, torch):
    """The 64-program batch under each `should_try_steal` policy (FixedWork, Greedy, LatencyBudget;
    Sec. 6), with persistent shares and with cluster launch control, beside the claim-cursor
    batch at the same launch shape.  LatencyBudget's budget is half of FixedWork's time."""
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    sizes = P.batch_sizes()
    ctx = gx.Context(torch.cuda.current_device())
    items = build_batch(gx, torch, ctx, sizes)
    total = sum(sizes)
    shape = (256, 4)

    def timed(b):
        for _ in range(2):
            b.launch(stream=sid)
        ts = []
        for _ in range(5):
            t = EventTimer(stream)
            with t:
                b.launch(stream=sid)
            ts.append(t.ms())
        return float(np.median(ts))

    out = {"workload": f"64 generated programs over log-uniform batches 4K-16M, {total} events",
           "launch": {"block": shape[0], "ept": shape[1]}}
    b = gx.Batch(ctx)
    for prog, _, dev, n in items:
        b.add(prog, dev, n)
    b.plan(launch=shape, stream=sid)
    ms = timed(b)
    out["claim_cursor"] = {"ms": round(ms, 3), "Mevents_per_s": round(total / ms / 1e3, 1)}
    b.destroy()
    for lc in (False, True):
        budget_ns = 0
        for kind in ("fixed", "greedy", "latency_budget"):
            hook, hspecs, cs = P.sched_policy(kind)
            hm = [gx.Map.from_spec(ctx, s) for s in hspecs]
            hp = gx.Program(ctx, hook, hm, cs, jit=True)
            b = gx.Batch(ctx)
            for prog, _, dev, n in items:
                b.add(prog, dev, n)
            b.set_sched(hp, budget_ns, launch_control=lc)
            b.plan(launch=shape, stream=sid)
            ms = timed(b)
            tally = b.sched_tally(stream=sid)
            if kind == "fixed":
                budget_ns = int(ms * 1e6 / 2)
            out[("launch_control_" if lc else "shares_") + kind] = {
                "ms": round(ms, 3), "Mevents_per_s": round(total / ms / 1e3, 1), "blocks": int(len(tally)),
                "stolen": int(tally[:, gx.STEAL_STOLEN].sum()), "asked": int(tally[:, gx.STEAL_ASKED].sum()),
                "budget_ns": budget_ns if kind == "latency_budget" else None, "status": int(hp.status().status)}
            b.destroy()
            hp.destroy()
            for m in hm:
                m.destroy()
    for prog, maps, dev, n in items:
        prog.destroy()
        for m in maps:
            m.destroy()
    ctx.close()
    return out


def run_warp(gx, torch, steps: int, warmup: int, n_warps: int = 1 << 21):
    """warp_heat over warp-context records (the warp-level form: one handler per warp, the leader's
    side effects once), page-heat beside it at the same record count and launch shape.  Both read
    32 B per record; roofline against the measured copy bandwidth."""
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    n = n_warps * 32
    ctx = gx.Context(torch.cuda.current_device())
    shape = (256, 8)
    out = {"workload": f"{n_warps} warps x 32 lanes of warp-context records (75% coalesced, Zipf(1.1) pages)",
           "events": n, "launch": {"block": shape[0], "ept": shape[1]}, "l2": "inputs 2 GiB per step > 129 MB L2"}
    peak, peak_kind = peaks()
    ev = gen.warp_access_events(n_warps)
    dev = to_device(ev)
    for name, build, simt in (("warp_heat", P.warp_heat, {"uniform": gen.WARP_UNIFORM}),
                              ("page_heat", P.page_heat, None)):
        prog_i, specs, cs = build()
        maps = [gx.Map.from_spec(ctx, sp) for sp in specs]
        prog = gx.Program(ctx, prog_i, maps, cs, deterministic=True, jit=True, simt=simt)
        for _ in range(max(3, warmup)):
            prog.run(dev, n, launch=shape, stream=sid)
        ts = []
        for _ in range(max(1, steps)):
            t = EventTimer(stream)
            with t:
                prog.run(dev, n, launch=shape, stream=sid)
            ts.append(t.ms())
        st = prog.status()
        ms = float(np.median(ts))
        achieved = n * 32 / (ms / 1e3) / 1e9
        out[name] = {"ms": round(ms, 4), "Mevents_per_s": round(n / ms / 1e3, 1), "status": int(st.status),
                     "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                                  "frac": round(achieved / peak, 4), "peak_kind": peak_kind}}
        prog.destroy()
        for m in maps:
            m.destroy()
    del dev
    ctx.close()
    return out


def run_served(gx, torch, seconds: float, lam: float = 20000.0):
    ctx = gx.Context(torch.cuda.current_device())
    rng = np.random.default_rng(SEED)
    progs = P.batch_programs()
    loaded = []
    for prog_i, specs, cs in progs:
        maps = [gx.Map.from_spec(ctx, s) for s in specs]
        loaded.append((gx.Program(ctx, prog_i, maps, cs, deterministic=True, jit=True), maps))
    n_req = int(lam * seconds)
    gaps = rng.exponential(1.0 / lam, n_req)
    offs = np.cumsum(gaps)
    lo, hi = math.log(1024), math.log(4 << 20)
    sizes = np.exp(lo + rng.random(n_req) * (hi - lo)).astype(np.int64)
    which = rng.integers(0, 64, n_req)
    pool_n = 4 << 20
    pool = to_device(gen.uniform_events(pool_n + (1 << 20), seed=SEED))  # request batches are slices of a pool
    starts = rng.integers(0, 1 << 20, n_req) * 32
    res = {}
    for mode in ("plain", "served"):
        srv = gx.Server(ctx, mem_budget=8 << 30, max_inflight=4, max_items=4096, block=256, ept=4,
                        plain=(mode == "plain"), progs=[p for p, _ in loaded])
        reqs = [(loaded[int(w)][0], pool.data_ptr() + int(s), int(n), None, i, float(o))
                for i, (w, s, n, o) in enumerate(zip(which, starts, sizes, offs))]
        done = []
        collector_stop = threading.Event()

        def collect():
            while not collector_stop.is_set() or len(done) < n_req:
                done.extend(srv.poll(8192, wait_ms=5))
                if collector_stop.is_set() and len(done) >= n_req:
                    break

        th = threading.Thread(target=collect, daemon=True)
        th.start()
        t0 = time.perf_counter()
        srv.replay(reqs)
        collector_stop.set()
        th.join(timeout=120)
        wall = time.perf_counter() - t0
        lat = np.array([c.t_done - c.t_arrival for c in done]) * 1e3
        first = min(c.t_arrival for c in done)
        last = max(c.t_done for c in done)
        ev_total = int(sizes.sum())
        res[mode] = {"requests": len(done), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                     "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
                     "Mevents_per_s": round(ev_total / (last - first) / 1e6, 1), "wall_s": round(wall, 2)}
        srv.destroy()
    out = {"workload": f"Poisson {lam:.0f} req/s for {seconds:.1f} s, 1K-4M events log-uniform, 64 programs, "
                       "8 GiB admission budget, maps resident",
           **res}
    for p, maps in loaded:
        p.destroy()
        for m in maps:
            m.destroy()
    ctx.close()
    return out


# ---------------------------------------------------------------------------- reference arm
# how page-heat's maps combine when the oracle runs parts of a batch in parallel, read off the
# program's definition: heat[region] = {count += w, last_ts = max(ts)} inserted as zeros, and
# the tally's two counters add
PAGEHEAT_ORACLE_MERGE = [{"words": [(0, 8, "add"), (8, 8, "max")], "insert": bytes(16)},
                         {"words": [(0, 8, "add"), (8, 8, "add")]}]


def oracle_pageheat_seconds(ev, threads):
    """Wall seconds of the oracle over `ev` on `threads` host threads (parts merged after)."""
    import oracle as O

    prog_i, specs, cs = P.page_heat()
    t0 = time.perf_counter()
    if threads == 1:
        O.run(prog_i, O.maps_from_specs(specs), ev, cs)
    else:
        O.run_parallel(prog_i, specs, ev, cs, PAGEHEAT_ORACLE_MERGE, threads=threads)
    return time.perf_counter() - t0


def reference_arm(args, rank, world):
    """The oracle as it stands, on the host cores (one thread per core, parts of each step
    merged), on bounded samples of the workload."""
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    n_sample = 1 << 23
    ev = gen.pageheat_events(n_sample, seed=SEED)
    oracle_pageheat_seconds(ev[:4096], cores)
    for _ in range(max(1, args.warmup)):
        oracle_pageheat_seconds(ev, cores)
    times = [oracle_pageheat_seconds(ev, cores) for _ in range(max(1, args.steps))]
    s = sum(times) / len(times)
    value = n_sample / s / 1e6
    line = {"metric": "page-heat throughput", "value": round(value, 3), "unit": "Mevents/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(s * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic", "impl": "reference",
            "config": {"workload": PAGEHEAT_WORKLOAD, "events_per_gpu": C2_EVENTS, "ctx_bytes": 32,
                       "sample_events_per_step": n_sample},
            "cpu_baseline": {"value": round(value, 3), "unit": "Mevents/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {n_sample} events of the 64M-event page-heat batch per step, "
                                       f"{cores} contiguous parts on {cores} threads, maps merged"},
            "e2e": {"value": round(value, 3), "unit": "Mevents/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample():
    """Oracle throughput on bounded samples of the headline workload: on every host core
    (contiguous parts on one thread each, maps merged), and on one core."""
    cores = os.cpu_count() or 1
    n, n1 = 16 << 20, 4 << 20
    ev = gen.pageheat_events(n, seed=SEED)
    s = oracle_pageheat_seconds(ev, cores)
    s1 = oracle_pageheat_seconds(ev[:n1], 1)
    return {"value": round(n / s / 1e6, 3), "unit": "Mevents/s", "cores": cores, "kind": "oracle",
            "sample": f"first {n} events of the 64M-event page-heat batch, {cores} parts on {cores} threads, "
                      f"maps merged ({s:.1f} s wall)",
            "single_core": {"value": round(n1 / s1 / 1e6, 3), "cores": 1,
                            "sample": f"first {n1} events on one thread ({s1:.1f} s)"}}


# ---------------------------------------------------------------------------- main
def main() -> int:
    global C2_EVENTS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--only", default="all", choices=["all", "headline", "latency", "batched", "served", "sched",
                                                      "warp"],
                    help="all / the headline line only / one config alone (for profiling); sched: the "
                         "64-program batch under each scheduling policy; warp: warp_heat's warp-level form "
                         "beside page-heat (neither part of the default line)")
    ap.add_argument("--pairs", type=int, default=C3_PAIRS, help="latency pairs with --only latency")
    ap.add_argument("--serve-rate", type=float, default=20000.0, help="served config arrival rate (req/s)")
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--events", type=int, default=C2_EVENTS, help="headline batch size (smaller for profiling)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    C2_EVENTS = args.events
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2512_12615_gb300 as gx

    gx.lib()
    if args.only in ("latency", "batched", "served", "sched", "warp"):
        one = {"latency": lambda: run_latency(gx, torch, True, args.pairs), "batched": lambda: run_batched(gx, torch),
               "served": lambda: run_served(gx, torch, args.serve_seconds, args.serve_rate),
               "sched": lambda: run_sched(gx, torch),
               "warp": lambda: run_warp(gx, torch, args.steps, args.warmup)}[args.only]()
        if rank == 0:
            print(json.dumps({"config": args.only, **one}), flush=True)
        return 0
    head = run_headline(args, gx, torch, (rank, world), jit=True)
    configs = {}
    if rank == 0:
        try:
            it = run_headline(args, gx, torch, (rank, world), jit=False)
            configs["page_heat_interpreter"] = {k: it[k] for k in ("value", "ms_per_step", "roofline", "launch_shape",
                                                                   "Minsns_per_s", "parity")}
        except Exception as e:
            configs["page_heat_interpreter"] = {"error": repr(e)}
    cpu = None
    if rank == 0 and args.only == "all":
        for name, fn in (("counting_1M", lambda: run_counting(gx, torch, True)),
                         ("counting_1M_interpreter", lambda: run_counting(gx, torch, False)),
                         ("latency_256M", lambda: run_latency(gx, torch, True)),
                         ("latency_256M_interpreter", lambda: run_latency(gx, torch, False)),
                         ("batched_64_programs", lambda: run_batched(gx, torch)),
                         ("served_poisson", lambda: run_served(gx, torch, args.serve_seconds, args.serve_rate)),
                         ("served_poisson_2k", lambda: run_served(gx, torch, args.serve_seconds, 2000.0))):
            try:
                configs[name] = fn()
            except Exception as e:  # a failing extra must not hide the headline
                configs[name] = {"error": repr(e)}
            torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = cpu_baseline_sample()
    if rank == 0:
        line = {"metric": "page-heat throughput", "value": head["value"], "unit": "Mevents/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
                "data": "synthetic", "exec": "jit (load-time specialised program; interpreter under configs)",
                "config": {"workload": PAGEHEAT_WORKLOAD,
                           "events_per_gpu": C2_EVENTS, "ctx_bytes": 32, "l2": "inputs 2 GiB per step > 129 MB L2",
                           "launch": head["launch_shape"], "maps": "resident across steps"},
                "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": head["e2e"], "clocks": head["clocks"],
                "gpu_launches": head["gpu_launches"], "insns_per_event": head["insns_per_event"],
                "Minsns_per_s": head["Minsns_per_s"],
                "Mevents_per_s_geomean_steps": head["Mevents_per_s_geomean_steps"], "parity": head["parity"],
                "configs": configs}
        print(json.dumps(line), flush=True)
        # a full-size result that differs from its closed form fails the run
        checked = [head["parity"]] + [c["parity"] for c in configs.values() if isinstance(c, dict) and "parity" in c]
        if not all(c["ok"] for c in checked):
            return 1
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
