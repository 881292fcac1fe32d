"""Engine vs oracle parity on the GPU, through the C ABI (bit-exact: integer results).

Sizes span many warps/blocks and end on ragged tails; every workload program, every
hand-worked program and all 64 generated batch programs are covered, under several
launch shapes.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from tests import closed_forms as CF
from tests.asmtext import assemble
from tests.parity import device_events, gpu_maps, run_both, snapshot_gpu
from workloads import gen
from workloads import programs as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    import paper_2512_12615_gb300 as gx

    c = gx.Context(0)
    yield c


def test_counting_parity(ctx):
    prog, specs, cs = P.counting()
    ev = gen.uniform_events(100_003, seed=21)
    gs, _, r0, _ = run_both(ctx, prog, specs, cs, ev)
    assert np.array_equal(gs[0][1].view("<u8")[:, 0], CF.counting(ev))


@pytest.mark.parametrize("launch", [(32, 1), (64, 3), (128, 2), (256, 1), (256, 16)])
def test_counting_launch_shapes(ctx, launch):
    prog, specs, cs = P.counting(n_counters=16)
    ev = gen.uniform_events(50_001, seed=22)
    run_both(ctx, prog, specs, cs, ev, launch=launch)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 255, 257, 32 * 257 + 5])
def test_ragged_sizes(ctx, n):
    prog, specs, cs = P.page_heat(max_entries=4096)
    run_both(ctx, prog, specs, cs, gen.pageheat_events(n, seed=23 + n))


def test_empty_batch(ctx):
    import paper_2512_12615_gb300 as gx

    prog, specs, cs = P.counting()
    m = gpu_maps(ctx, specs)
    p = gx.Program(ctx, prog, m, cs)
    dev = torch.zeros(16, dtype=torch.uint8, device="cuda")
    p.run(dev, 0)
    torch.cuda.synchronize()
    assert m[0].array_u64().sum() == 0


def test_page_heat_parity(ctx):
    prog, specs, cs = P.page_heat()
    ev = gen.pageheat_events(200_001, seed=24)
    ev["size"][::97] = 3
    ev["kind"][5::101] = 9
    ev["addr"][7::89] |= np.uint64(1)
    gs, _, _, _ = run_both(ctx, prog, specs, cs, ev)
    heat, tally = CF.page_heat(ev)
    got = {int.from_bytes(k, "little"): (int.from_bytes(v[:8], "little"), int.from_bytes(v[8:], "little"))
           for k, v in gs[0][1].items()}
    assert got == heat


def test_latency_parity(ctx):
    prog, specs, cs = P.latency(ring_bytes=1 << 22)
    ev = gen.latency_pairs(100_001, seed=25)
    ev["kind"][6] = 5
    gs, os_, _, _ = run_both(ctx, prog, specs, cs, ev)
    hist, outliers = CF.latency(ev)
    assert np.array_equal(gs[0][1].view("<u8")[:, 0], hist)
    assert gs[1][1] == outliers and gs[1][2] == 0


@pytest.mark.parametrize("p", range(64))
def test_random_program_parity(ctx, p):
    progs = P.batch_programs()
    prog, specs, cs = progs[p]
    run_both(ctx, prog, specs, cs, gen.uniform_events(20_000 + 37 * p, seed=300 + p))


@pytest.mark.parametrize("p", [0, 17, 42, 63])
@pytest.mark.parametrize("launch", [(64, 1), (256, 8)])
def test_random_program_shapes(ctx, p, launch):
    prog, specs, cs = P.batch_programs()[p]
    run_both(ctx, prog, specs, cs, gen.pageheat_events(9_999, seed=400 + p), launch=launch)


CASES = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "handworked.json")))["cases"]


GPU_CASES = [c for c in CASES if "oracle_only" not in c]  # the others state why the engine cannot run them


@pytest.mark.parametrize("case", GPU_CASES, ids=[c["name"] for c in GPU_CASES])
def test_handworked_on_gpu(ctx, case):
    """The hand-derived expectations hold on the engine too (rings enlarged to the 4 KiB minimum)."""
    if case["name"] == "ringbuf_full_drops":
        pytest.skip("needs a 64-byte ring; covered by test_ringbuf_drops")
    specs = [dict(m) for m in case.get("maps", [])]
    for m in specs:
        if m["type"] == 27:
            m["max_entries"] = max(4096, m["max_entries"])
    ev = np.array(case["events"], dtype=np.uint64)
    gs, _, r0, _ = run_both(ctx, assemble(case["asm"]).prog(), specs, 8 * ev.shape[1], ev, det=False)
    exp = case["expect"]
    assert r0.tolist() == exp["r0"]
    for idx, words in exp.get("array_u64", {}).items():
        assert gs[int(idx)][1].view("<u8")[:, 0].tolist() == words
    for idx, recs in exp.get("ring", {}).items():
        assert [(i, p.hex()) for i, p in gs[int(idx)][1]] == [tuple(r) for r in recs]


def test_ringbuf_drops(ctx):
    """A 4 KiB ring holds 64 records of 16 + 48 bytes; later reservations fail and count."""
    import paper_2512_12615_gb300 as gx

    lines = ["mov r6 r1", "ld_map r1 0", "mov r2 48", "mov r3 0", "call ringbuf_reserve", "jeq r0 0 out",
             "ldx8 r2 r6 0", "stx8 r0 40 r2", "mov r1 r0", "mov r2 0", "call ringbuf_submit", "mov r0 1", "exit",
             "out:", "exit"]
    specs = [dict(type=27, key_size=0, value_size=0, max_entries=4096)]
    ev = np.zeros((1000, 2), dtype=np.uint64)
    ev[:, 0] = np.arange(1000)
    m = gpu_maps(ctx, specs)
    p = gx.Program(ctx, assemble(lines).prog(), m, 16)
    ret = torch.zeros(1000, dtype=torch.int64, device="cuda")
    p.run(device_events(ev), 1000, ret_out=ret)
    raw, dropped = m[0].drain()
    recs = gx.parse_records(raw)
    assert len(recs) == 64 and dropped == 1000 - 64
    assert int(ret.sum()) == 64
    idx = {i for i, _ in recs}
    assert all(int.from_bytes(pl[40:48], "little") == i for i, pl in recs) and len(idx) == 64
    # drained: the next run starts from an empty ring
    p.run(device_events(ev[:10]), 10)
    raw, dropped = m[0].drain()
    assert len(gx.parse_records(raw)) == 10 and dropped == 0


def _mixed_ring_program():
    """Reserves 8, 48 or 200 payload bytes (records of 24, 64 and 216 bytes) by ctx word 1,
    writes ctx word 0 into the payload, submits; R0 = 1 if the reservation succeeded."""
    lines = ["mov r6 r1", "ldx8 r8 r6 0", "ldx8 r7 r6 8", "jeq r7 0 mid", "jeq r7 1 big"]
    for label, size in ((None, 8), ("mid", 48), ("big", 200)):
        lines += ([f"{label}:"] if label else []) + [
            "ld_map r1 0", f"mov r2 {size}", "mov r3 0", "call ringbuf_reserve", "jeq r0 0 out", "stx8 r0 0 r8",
            "mov r1 r0", "mov r2 0", "call ringbuf_submit", "mov r0 1", "exit"]
    return assemble(lines + ["out:", "exit"]).prog()


@pytest.mark.parametrize("jit", [False, True])
def test_ringbuf_mixed_sizes_overflow(ctx, jit):
    """Mixed record sizes into an 8 KiB ring, 3,000 events: the ring closes at the first record
    that does not fit (the oracle's rule), so what the device keeps is a valid outcome of a
    concurrent run.  Against the oracle with a ring large enough for everything: every kept
    record is one of its records, byte for byte; kept + dropped = all of them; R0 says which
    were kept; the kept records fill the ring to within one largest record.  The oracle's own
    8 KiB run obeys the same bounds."""
    import paper_2512_12615_gb300 as gx

    cap, n = 8192, 3000
    prog = _mixed_ring_program()
    rng = np.random.default_rng(0x51)
    ev = np.zeros((n, 2), dtype=np.uint64)
    ev[:, 0] = rng.integers(1, 1 << 62, n, dtype=np.uint64)
    ev[:, 1] = rng.integers(0, 3, n)
    rec_of = {0: 64, 1: 216, 2: 24}
    om = O.maps_from_specs([dict(type=27, key_size=0, value_size=0, max_entries=1 << 20)])
    r0_all, _ = O.run(prog, om, ev, 16, want_r0=True)
    every, d_all = om[0].ringbuf_records()
    assert d_all == 0 and len(every) == n and all(int(x) == 1 for x in r0_all)
    every = dict(every)
    ob = O.maps_from_specs([dict(type=27, key_size=0, value_size=0, max_entries=cap)])
    r0_o, _ = O.run(prog, ob, ev, 16, want_r0=True)
    kept_o, dropped_o = ob[0].ringbuf_records()
    used_o = sum(rec_of[int(ev[i, 1])] for i, _ in kept_o)
    assert [i for i, _ in kept_o] == list(range(len(kept_o)))  # sequential: a prefix, then closed
    assert len(kept_o) + dropped_o == n and cap - 216 < used_o <= cap
    m = gpu_maps(ctx, [dict(type=27, key_size=0, value_size=0, max_entries=cap)])
    p = gx.Program(ctx, prog, m, 16, jit=jit)
    ret = torch.zeros(n, dtype=torch.int64, device="cuda")
    p.run(device_events(ev), n, ret_out=ret)
    assert p.status().status == 0
    raw, dropped = m[0].drain()
    recs = gx.parse_records(raw)
    idx = [i for i, _ in recs]
    assert len(set(idx)) == len(idx)
    assert all(every[i] == pl for i, pl in recs)
    assert len(recs) + dropped == n
    r0 = ret.cpu().numpy()
    assert set(np.nonzero(r0 == 1)[0].tolist()) == set(idx) and set(np.unique(r0).tolist()) <= {0, 1}
    used = sum(rec_of[int(ev[i, 1])] for i in idx)
    assert cap - 216 < used <= cap
    p.destroy()
    m[0].destroy()


def test_budget_trip_is_reported_not_hung(ctx):
    import paper_2512_12615_gb300 as gx

    lines = ["mov r0 0", "mov r2 0", "l:", "add r0 1", "add r2 1", "jlt r2 5000 l", "exit"]
    p = gx.Program(ctx, assemble(lines).prog(), [], 16, insn_budget=100)
    ev = np.zeros((77, 2), dtype=np.uint64)
    ret = torch.full((77,), 7, dtype=torch.int64, device="cuda")
    p.run(device_events(ev), 77, ret_out=ret)
    st = p.status(reset=True)
    assert st.status == gx.E_BUDGET and st.budget_trips == 77
    assert int(ret.abs().sum()) == 0
    p2 = gx.Program(ctx, assemble(lines).prog(), [], 16)
    p2.run(device_events(ev), 77, ret_out=ret)
    assert p2.status().status == 0 and ret.tolist() == [5000] * 77


def test_divergent_loops_reconverge(ctx):
    """Per-event trip counts differ inside a warp: min-pc scheduling must still finish all."""
    lines = ["ldx8 r2 r1 0", "and r2 63", "mov r0 0", "jeq r2 0 done", "l:", "add r0 r2", "add r2 -1",
             "jne r2 0 l", "done:", "exit"]
    ev = np.zeros((5000, 2), dtype=np.uint64)
    ev[:, 0] = np.random.default_rng(1).integers(0, 1 << 40, 5000)
    _, _, r0, _ = run_both(ctx, assemble(lines).prog(), [], 16, ev, det=False)
    k = (ev[:, 0] & 63).astype(np.int64)
    assert np.array_equal(r0, k * (k + 1) // 2)


def test_map_snapshot_restore(ctx):
    import paper_2512_12615_gb300 as gx

    h = gx.Map(ctx, gx.MAP_HASH, 8, 16, 1000)
    pairs = b"".join(int(k).to_bytes(8, "little") + int(3 * k).to_bytes(8, "little") + int(k + 1).to_bytes(8, "little")
                     for k in range(700))
    h.write(pairs)
    items = h.hash_items()
    assert len(items) == 700 and items[(5).to_bytes(8, "little")] == (15).to_bytes(8, "little") + (6).to_bytes(8, "little")
    h.clear()
    assert h.hash_items() == {}
    a = gx.Map(ctx, gx.MAP_ARRAY, 4, 12, 33)
    vals = bytes(range(256)) * 2
    a.write(vals[:33 * 12])
    assert a.array_values().tobytes() == vals[:33 * 12]


def test_hash_capacity_on_gpu(ctx):
    """More distinct keys than max_entries: exactly max_entries live keys, all correct."""
    import paper_2512_12615_gb300 as gx

    prog, specs, cs = P.page_heat(max_entries=512)
    ev = gen.pageheat_events(100_000, seed=26)
    gm = gpu_maps(ctx, specs)
    p = gx.Program(ctx, prog, gm, cs, deterministic=True)
    p.run(device_events(ev), len(ev))
    torch.cuda.synchronize()
    got = gm[0].hash_items()
    heat, _ = CF.page_heat(ev)
    assert len(heat) > 512 and len(got) == 512
    for k, v in got.items():  # surviving keys carry exactly their totals
        assert (int.from_bytes(v[:8], "little"), int.from_bytes(v[8:], "little")) == heat[int.from_bytes(k, "little")]


def test_autotune_leaves_maps_untouched(ctx):
    import paper_2512_12615_gb300 as gx

    prog, specs, cs = P.counting()
    ev = gen.uniform_events(300_000, seed=27)
    gm = gpu_maps(ctx, specs)
    p = gx.Program(ctx, prog, gm, cs)
    dev = device_events(ev)
    block, ept, _ = p.autotune(dev, len(ev))
    assert block in (128, 256) and ept >= 1
    assert gm[0].array_u64().sum() == 0
    p.run(dev, len(ev))
    assert np.array_equal(gm[0].array_u64()[:, 0], CF.counting(ev))


def test_host_buffer_path_matches(ctx):
    import paper_2512_12615_gb300 as gx

    prog, specs, cs = P.page_heat()
    ev = gen.pageheat_events(300_007, seed=28)
    gm = gpu_maps(ctx, specs)
    p = gx.Program(ctx, prog, gm, cs, deterministic=True)
    ret = np.zeros(len(ev), dtype=np.int64)
    p.run_host(ev, ret)
    om = O.maps_from_specs(specs)
    r0_o, _ = O.run(prog, om, ev, cs, want_r0=True)
    assert np.array_equal(ret, r0_o)
    assert gm[0].hash_items() == om[0].hash_items()


@pytest.mark.parametrize("jit", [False, True])
@pytest.mark.parametrize("pinned_ret", [False, True])
def test_host_buffer_path_pinned(ctx, jit, pinned_ret):
    """Page-locked host buffers for the events and for R0 (or a pageable R0 buffer) through the
    staged host path."""
    import paper_2512_12615_gb300 as gx

    prog, specs, cs = P.page_heat()
    ev = gen.pageheat_events(250_001, seed=29)
    pinned = torch.empty(ev.nbytes, dtype=torch.uint8).pin_memory()
    pinned.numpy()[:] = ev.view(np.uint8).reshape(-1)
    gm = gpu_maps(ctx, specs)
    p = gx.Program(ctx, prog, gm, cs, deterministic=True, jit=jit)
    if pinned_ret:
        ret_t = torch.zeros(len(ev), dtype=torch.int64).pin_memory()
        ret = ret_t.numpy()
    else:
        ret = np.zeros(len(ev), dtype=np.int64)
    p.run_host(pinned.numpy().view(ev.dtype), ret)
    om = O.maps_from_specs(specs)
    r0_o, _ = O.run(prog, om, ev, cs, want_r0=True)
    assert np.array_equal(ret, r0_o)
    assert gm[0].hash_items() == om[0].hash_items()
    assert p.status().status == 0


def test_verify_load_rejection_raises(ctx):
    import paper_2512_12615_gb300 as gx

    with pytest.raises(gx.GxError) as e:
        gx.Program(ctx, assemble(["ldx8 r0 r10 -8", "exit"]).prog(), [], 16)
    assert e.value.status == gx.E_VERIFY and "uninitialised stack" in e.value.log
