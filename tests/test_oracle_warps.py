"""Pins the oracle's warp (lockstep) run, the warp-level execution of Sec. 4.4.1 / Sec. 4.4.2.

Against what fixes it independently of its own code:
- one lane per warp is the sequential run (one handler execution per event);
- warps of identical lanes are one sequential execution per warp;
- the warp helpers are the numpy reductions over each warp's lanes (ragged last warp);
- each disagreement the definition names (a branch, a map key, an atomic or store into
  shared memory, a helper payload, R0 at exit) stops the run at that instruction, and a
  value aggregated first does not.
"""
import numpy as np
import pytest

import oracle as O
from tests.asmtext import assemble
from workloads import gen
from workloads import programs as P


def snapshot(maps):
    out = []
    for m in maps:
        if m.type == O.MAP_HASH:
            out.append(sorted(m.hash_items().items()))
        elif m.type == O.MAP_ARRAY:
            out.append(m.array_values().tobytes())
        else:
            out.append(m.ringbuf_records())
    return out


def workload_cases():
    yield "counting", P.counting(), gen.uniform_events(3_001, seed=1)
    yield "page_heat", P.page_heat(), gen.pageheat_events(3_001, seed=2)
    yield "latency", P.latency(ring_bytes=1 << 16), gen.latency_pairs(2_001, seed=3)
    for p in (0, 9, 17, 33, 42, 63):
        yield f"random{p}", P.batch_programs()[p], gen.uniform_events(1_001, seed=100 + p)


@pytest.mark.parametrize("name,pc,ev", list(workload_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_one_lane_is_the_sequential_run(name, pc, ev):
    prog, specs, cs = pc
    m_seq, m_warp = O.maps_from_specs(specs), O.maps_from_specs(specs)
    r_seq, c_seq = O.run(prog, m_seq, ev, cs, want_r0=True)
    r_warp, c_warp = O.run_warps(prog, m_warp, ev, cs, lanes=1, want_r0=True)
    assert np.array_equal(r_seq, r_warp) and c_seq == c_warp
    assert snapshot(m_seq) == snapshot(m_warp)


@pytest.mark.parametrize("lanes", [2, 7, 32])
@pytest.mark.parametrize("name,pc,ev", list(workload_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_identical_lanes_are_one_execution_per_warp(name, pc, ev, lanes):
    prog, specs, cs = pc
    ev = ev[:300]
    raw = np.ascontiguousarray(ev).view(np.uint8).reshape(-1, cs)  # one row per ctx
    rep = np.repeat(raw, lanes, axis=0)  # warp i = `lanes` byte copies of event i
    m_seq, m_warp = O.maps_from_specs(specs), O.maps_from_specs(specs)
    r_seq, c_seq = O.run(prog, m_seq, ev, cs, want_r0=True)
    r_warp, c_warp = O.run_warps(prog, m_warp, rep, cs, lanes=lanes, want_r0=True,
                                 uniform=np.ones(cs, dtype=bool))
    assert np.array_equal(np.repeat(r_seq, lanes), r_warp) and c_seq == c_warp
    seq, warp = snapshot(m_seq), snapshot(m_warp)
    for m, a, b in zip(specs, seq, warp):
        if m["type"] == O.MAP_RINGBUF:  # a record carries its warp leader's event index
            assert [(i * lanes, p) for i, p in a[0]] == b[0] and a[1] == b[1]
        else:
            assert a == b


REDUCE = {
    "warp_sum_u64": lambda v: int(v.sum(dtype=np.uint64)),
    "warp_max_u64": lambda v: int(v.max()),
    "warp_min_u64": lambda v: int(v.min()),
    "warp_or_u64": lambda v: int(np.bitwise_or.reduce(v)),
    "warp_and_u64": lambda v: int(np.bitwise_and.reduce(v)),
    "warp_count": lambda v: int((v != 0).sum()),
}


@pytest.mark.parametrize("helper", sorted(REDUCE))
@pytest.mark.parametrize("lanes,n", [(32, 70), (5, 23), (1, 4)])
def test_warp_helpers_are_reductions(helper, lanes, n):
    rng = np.random.default_rng(lanes * 1000 + n)
    ev = np.zeros((n, 2), dtype=np.uint64)
    ev[:, 0] = rng.integers(0, 2**64 - 1, size=n, dtype=np.uint64, endpoint=True)
    ev[rng.random(n) < 0.3, 0] = 0  # zeros for the count
    ev[:, 0][ev[:, 0] > 2**63] |= np.uint64(1)  # sums that wrap
    prog = assemble(["ldx8 r1 r1 0", f"call {helper}", "exit"]).prog()
    r0, _ = O.run_warps(prog, [], ev, 16, lanes=lanes, want_r0=True)
    for w0 in range(0, n, lanes):
        want = REDUCE[helper](ev[w0:w0 + lanes, 0])
        assert [int(x) & (2**64 - 1) for x in r0[w0:w0 + lanes]] == [want] * len(ev[w0:w0 + lanes])


def test_warp_helpers_are_not_part_of_the_per_event_run():
    with pytest.raises(O.OracleError) as e:
        O.run(assemble(["mov r1 1", "call warp_sum_u64", "exit"]).prog(), [], np.zeros((1, 2), np.uint64), 16)
    assert e.value.rc == O.EINVAL


# ctx: word 0 = region (uniform), word 1 = lane address (varying)
UNI = np.array([True] * 8 + [False] * 8)
ARR = [dict(type=2, key_size=4, value_size=8, max_entries=4)]
HASH = [dict(type=1, key_size=8, value_size=8, max_entries=64)]
RING = [dict(type=27, key_size=0, value_size=0, max_entries=4096)]


def warp_events(lanes, warps, seed, vary=True):
    rng = np.random.default_rng(seed)
    ev = np.zeros((lanes * warps, 2), dtype=np.uint64)
    ev[:, 0] = np.repeat(rng.integers(0, 4, size=warps), lanes)
    ev[:, 1] = rng.integers(0, 1 << 40, size=lanes * warps) if vary else np.repeat(rng.integers(0, 1 << 40, warps), lanes)
    return ev


def lookup0(reg_key="r7"):
    return [f"stx4 r10 -4 {reg_key}", "ld_map r1 0", "mov r2 r10", "add r2 -4", "call map_lookup_elem"]


DIVERGING = {  # (program, maps, index of the slot where the lanes disagree; ld_map takes two)
    # a branch on the lane address
    "branch": (["ldx8 r7 r1 8", "and r7 1", "mov r0 0", "jeq r7 0 out", "mov r0 1", "out:", "exit"], [], 3),
    # the lane address as an update key
    "key": (["ldx8 r7 r1 8", "stx8 r10 -8 r7", "stx8 r10 -16 r7", "ld_map r1 0", "mov r2 r10", "add r2 -8",
             "mov r3 r10", "add r3 -16", "mov r4 0", "call map_update_elem", "mov r0 0", "exit"], HASH, 10),
    # a lane-varying operand added into a map value
    "atomic": (["ldx8 r6 r1 8", "ldx8 r7 r1 0"] + lookup0() + ["jeq r0 0 out", "atomic8 add r0 0 r6", "out:",
                                                                "mov r0 0", "exit"], ARR, 9),
    # a lane-varying value stored into a map value
    "store": (["ldx8 r6 r1 8", "ldx8 r7 r1 0"] + lookup0() + ["jeq r0 0 out", "stx8 r0 0 r6", "out:", "mov r0 0",
                                                               "exit"], ARR, 9),
    # a lane-varying ring-buffer payload
    "payload": (["ldx8 r6 r1 8", "stx8 r10 -8 r6", "ld_map r1 0", "mov r2 r10", "add r2 -8", "mov r3 8", "mov r4 0",
                 "call ringbuf_output", "mov r0 0", "exit"], RING, 8),
    # a lane-varying R0
    "exit": (["ldx8 r0 r1 8", "exit"], [], 1),
    # a lane-varying operand of the atomic max helper
    "atomic_max": (["ldx8 r6 r1 8", "ldx8 r7 r1 0"] + lookup0() + ["jeq r0 0 out", "mov r1 r0", "mov r2 r6",
                                                                    "call atomic_max_u64", "out:", "mov r0 0", "exit"],
                   ARR, 11),
}


@pytest.mark.parametrize("case", sorted(DIVERGING))
def test_disagreement_stops_the_warp(case):
    lines, specs, pc = DIVERGING[case]
    prog = assemble(lines).prog()
    ev = warp_events(32, 3, seed=len(case))
    with pytest.raises(O.OracleError) as e:
        O.run_warps(prog, O.maps_from_specs(specs), ev, 16, uniform=UNI)
    assert e.value.rc == O.EDIVERGE and e.value.pc == pc and e.value.event == 0
    # the same program over warps whose lanes agree runs through
    O.run_warps(prog, O.maps_from_specs(specs), warp_events(32, 3, seed=len(case), vary=False), 16, uniform=UNI)


def test_aggregated_then_used():
    """Lane-varying addresses reduced by warp_count, then added once per warp at a uniform key
    (the region): the map holds, per region, the number of odd addresses."""
    # the ctx pointer is kept in R9: R1..R5 are cleared by the call
    lines = ["mov r9 r1", "ldx8 r1 r9 8", "and r1 1", "call warp_count", "mov r6 r0", "ldx8 r7 r9 0"] + lookup0() + [
        "jeq r0 0 out", "atomic8 add r0 0 r6", "out:", "mov r0 0", "exit"]
    ev = warp_events(32, 40, seed=5)
    ev = np.concatenate([ev, warp_events(9, 1, seed=6)])  # ragged last warp
    m = O.maps_from_specs(ARR)
    r0, count = O.run_warps(assemble(lines).prog(), m, ev, 16, uniform=UNI, want_r0=True)
    want = np.zeros(4, dtype=np.uint64)
    np.add.at(want, ev[:, 0].astype(np.int64), ev[:, 1] & np.uint64(1))
    assert m[0].array_u64()[:, 0].tolist() == want.tolist()
    assert not r0.any() and count == 41 * 15  # 15 instructions per warp, the 64-bit immediate once


def test_stack_is_per_lane():
    """Stores and atomics on a lane's own stack stay lane-private: each lane keeps its address."""
    lines = ["ldx8 r6 r1 8", "stx8 r10 -8 r6", "mov r2 5", "atomic8 add r10 -8 r2", "ldx8 r6 r10 -8",
             "mov r1 r6", "call warp_sum_u64", "exit"]
    ev = warp_events(32, 2, seed=7)
    r0, _ = O.run_warps(assemble(lines).prog(), [], ev, 16, uniform=UNI, want_r0=True)
    for w in range(2):
        s = int((ev[32 * w:32 * (w + 1), 1] + np.uint64(5)).sum(dtype=np.uint64))
        assert r0[32 * w:32 * (w + 1)].tolist() == [s] * 32


def test_uniform_field_must_agree():
    ev = warp_events(4, 2, seed=8)
    ev[5, 0] += np.uint64(1)
    with pytest.raises(O.OracleError) as e:
        O.run_warps(assemble(["mov r0 0", "exit"]).prog(), [], ev, 16, uniform=UNI, lanes=4)
    assert e.value.rc == O.EINVAL and e.value.event == 4


def test_branch_that_agrees_is_fine():
    """Lanes may branch on a varying field when every lane goes the same way."""
    lines = DIVERGING["branch"][0]
    ev = warp_events(32, 2, seed=9)
    ev[:32, 1] &= ~np.uint64(1)
    ev[32:, 1] |= np.uint64(1)
    r0, _ = O.run_warps(assemble(lines).prog(), [], ev, 16, uniform=UNI, want_r0=True)
    assert r0.tolist() == [0] * 32 + [1] * 32


@pytest.mark.parametrize("lanes", [1, 3, 32])
def test_fetched_values_reach_every_lane(lanes):
    """A fetch-add and CMPXCHGs on a map value run once per warp, and every lane receives the
    old value.  Warp w (in order): the fetch-add returns w; a CMPXCHG expecting the current
    word 7w succeeds and stores 7w + 7; one expecting -1 fails and returns 7w + 7."""
    lines = (lookup0() + ["jeq r0 0 out", "mov r8 r0", "mov r3 1", "atomic8 add_fetch r8 0 r3",
                          "ldx8 r0 r8 8", "mov r4 r0", "add r4 7", "atomic8 cmpxchg r8 8 r4",
                          "mov r0 -1", "atomic8 cmpxchg r8 8 r4",
                          "lsh r0 32", "or r0 r3", "exit", "out:", "mov r0 -1", "exit"])
    lines = ["mov r7 0"] + lines
    specs = [dict(type=2, key_size=4, value_size=16, max_entries=1)]
    warps = 5
    ev = np.zeros((warps * lanes, 2), dtype=np.uint64)
    m = O.maps_from_specs(specs)
    r0, _ = O.run_warps(assemble(lines).prog(), m, ev, 16, uniform=np.ones(16, bool), lanes=lanes, want_r0=True)
    want = [((7 * w + 7) << 32) | w for w in range(warps)]
    assert r0.tolist() == np.repeat(want, lanes).tolist()
    assert m[0].array_u64()[0].tolist() == [warps, 7 * warps]
