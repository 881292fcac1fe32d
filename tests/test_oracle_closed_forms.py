"""Pins the oracle on the workload programs by closed forms, invariants and brute force.

* counting == bincount(kind); page_heat == group-by(addr >> 21); latency == 2-D histogram
  of (kernel id, floor log2 latency) plus the outlier list (closed forms in
  tests/closed_forms.py, computed with numpy straight from the event fields);
* a hash map and an array map fed the same keys give the same counts (brute force over
  a tiny key space);
* the random batch programs run without faults and their R0 does not depend on how the
  event range is split into calls (map state carries over, events are independent).
"""
import numpy as np
import pytest

import oracle as O
from tests import closed_forms as CF
from tests.asmtext import assemble
from workloads import gen
from workloads import programs as P


def test_counting_is_bincount():
    prog, specs, cs = P.counting()
    ev = gen.uniform_events(50_000, seed=11)
    maps = O.maps_from_specs(specs)
    r0, count = O.run(prog, maps, ev, cs, want_r0=True)
    assert np.array_equal(maps[0].array_u64()[:, 0], CF.counting(ev))
    assert np.array_equal(r0, ev["kind"].astype(np.int64))
    # 15 instructions per accepted event (straight-line path)
    assert count == 15 * len(ev)


def test_counting_bounds_check():
    prog, specs, cs = P.counting(n_counters=4)
    ev = gen.uniform_events(10_000, seed=12)
    maps = O.maps_from_specs(specs)
    O.run(prog, maps, ev, cs)
    assert np.array_equal(maps[0].array_u64()[:, 0], CF.counting(ev, 4))


def test_page_heat_is_groupby():
    prog, specs, cs = P.page_heat()
    ev = gen.pageheat_events(60_000, seed=13)
    # plant invalid and misaligned records so every branch is exercised
    ev["size"][::97] = 3
    ev["kind"][5::101] = 9
    ev["addr"][7::89] |= np.uint64(1)
    maps = O.maps_from_specs(specs)
    r0, _ = O.run(prog, maps, ev, cs, want_r0=True)
    heat, tally = CF.page_heat(ev)
    got = {int.from_bytes(k, "little"): (int.from_bytes(v[:8], "little"), int.from_bytes(v[8:], "little"))
           for k, v in maps[0].hash_items().items()}
    assert got == heat
    assert np.array_equal(maps[1].array_u64(), tally)


def test_latency_is_histogram():
    prog, specs, cs = P.latency(ring_bytes=1 << 22)
    ev = gen.latency_pairs(40_000, seed=14)
    ev["kind"][6] = 5  # a broken pair
    maps = O.maps_from_specs(specs)
    O.run(prog, maps, ev, cs)
    hist, outliers = CF.latency(ev)
    assert np.array_equal(maps[0].array_u64()[:, 0], hist)
    recs, dropped = maps[1].ringbuf_records()
    assert dropped == 0
    assert recs == outliers
    assert 0.005 < len(outliers) / 40_000 < 0.02  # about 1% by construction


def test_latency_zero_and_huge():
    """floor(log2) edge cases: latency 0 -> bucket 0, 1 -> 0, 2^63 -> 63."""
    prog, specs, cs = P.latency(n_kernels=4, ring_bytes=1 << 12)
    ev = gen.latency_pairs(3, seed=1, n_kernels=4)
    base = ev["ts_ns"][0]
    for j, lat in enumerate([0, 1, 1 << 63]):
        ev["ts_ns"][2 * j] = base
        ev["ts_ns"][2 * j + 1] = base + np.uint64(lat)
    maps = O.maps_from_specs(specs)
    O.run(prog, maps, ev, cs)
    hist, outliers = CF.latency(ev, n_kernels=4)
    assert np.array_equal(maps[0].array_u64()[:, 0], hist)
    kid = [int(ev["addr"][2 * j] & 0xFFFFFFFF) for j in range(3)]
    assert hist[kid[0] * 64 + 0] >= 1 and hist[kid[2] * 64 + 63] >= 1
    assert [i for i, _ in outliers] == [2]


HASH_COUNT = ["ldx4 r2 r1 0", "and r2 7", "stx8 r10 -8 r2",
              "ld_map r1 0", "mov r2 r10", "add r2 -8", "call map_lookup_elem", "jne r0 0 have",
              "st8 r10 -16 0",
              "ld_map r1 0", "mov r2 r10", "add r2 -8", "mov r3 r10", "add r3 -16", "mov r4 1",
              "call map_update_elem",
              "ld_map r1 0", "mov r2 r10", "add r2 -8", "call map_lookup_elem", "jeq r0 0 out",
              "have:", "mov r1 1", "atomic8 add r0 0 r1", "out:", "mov r0 0", "exit"]
ARRAY_COUNT = ["ldx4 r2 r1 0", "and r2 7", "stx4 r10 -4 r2",
               "ld_map r1 0", "mov r2 r10", "add r2 -4", "call map_lookup_elem", "jeq r0 0 out",
               "mov r1 1", "atomic8 add r0 0 r1", "out:", "mov r0 0", "exit"]


@pytest.mark.parametrize("seed", range(5))
def test_hash_and_array_agree_on_tiny_key_space(seed):
    rng = np.random.default_rng(seed)
    ev = np.zeros((200, 2), dtype=np.uint64)
    ev[:, 0] = rng.integers(0, 1 << 32, 200)
    hm = O.Map(O.MAP_HASH, 8, 8, 8)
    am = O.Map(O.MAP_ARRAY, 4, 8, 8)
    O.run(assemble(HASH_COUNT).prog(), [hm], ev, 16)
    O.run(assemble(ARRAY_COUNT).prog(), [am], ev, 16)
    h = {int.from_bytes(k, "little"): int.from_bytes(v, "little") for k, v in hm.hash_items().items()}
    a = am.array_u64()[:, 0]
    assert {k: v for k, v in enumerate(a.tolist()) if v} == h
    assert sum(h.values()) == 200
    assert a.tolist() == np.bincount((ev[:, 0] & 7).astype(np.int64), minlength=8).tolist()


def test_hash_capacity_limit():
    """Inserting 9 distinct keys into 8 entries: exactly 8 live keys, one insert refused."""
    hm = O.Map(O.MAP_HASH, 8, 8, 8)
    ev = np.zeros((9, 2), dtype=np.uint64)
    ev[:, 0] = np.arange(9)
    prog = assemble([l.replace("and r2 7", "and r2 15") for l in HASH_COUNT]).prog()
    O.run(prog, [hm], ev, 16)
    items = hm.hash_items()
    assert len(items) == 8 and 8 not in {int.from_bytes(k, "little") for k in items}


@pytest.mark.parametrize("p", range(0, 64, 9))
def test_random_programs_split_invariance(p):
    progs = P.batch_programs()
    prog, specs, cs = progs[p]
    ev = gen.uniform_events(3000, seed=100 + p)
    m1 = O.maps_from_specs(specs)
    r_all, _ = O.run(prog, m1, ev, cs, want_r0=True)
    m2 = O.maps_from_specs(specs)
    r_a, _ = O.run(prog, m2, ev[:1234], cs, want_r0=True)
    r_b, _ = O.run(prog, m2, ev[1234:], cs, want_r0=True, event_idx_base=1234)
    assert np.array_equal(r_all, np.concatenate([r_a, r_b]))
    assert np.array_equal(m1[0].array_values(), m2[0].array_values())
    assert m1[1].hash_items() == m2[1].hash_items()


def test_random_program_lengths():
    progs = P.batch_programs()
    lens = [len(p[0]) for p in progs]
    assert len(progs) == 64 and min(lens) >= 10 and max(lens) <= 400


def warp_heat_events(n_warps, seed, tail=13):
    """Warp-context records with planted bad warps (size 3, kind 9), misaligned lanes and a
    ragged last warp of `tail` lanes."""
    ev = gen.warp_access_events(n_warps, seed=seed)
    w = ev.reshape(n_warps, 32)
    w["size"][::37] = 3
    w["kind"][5::41] = 9
    w["addr"][3::7, 4::9] |= np.uint64(1)
    extra = gen.warp_access_events(1, seed=seed + 1)[:tail]
    return np.concatenate([ev, extra])


@pytest.mark.parametrize("seed", [21, 22])
def test_warp_heat_is_a_per_warp_groupby(seed):
    """The oracle's warp run of the warp-level policy equals its closed form: per warp the
    lowest / highest region, the lanes in the lowest, the sizes and the misaligned lanes."""
    prog, specs, cs = P.warp_heat()
    ev = warp_heat_events(1500, seed)
    maps = O.maps_from_specs(specs)
    r0, _ = O.run_warps(prog, maps, ev, cs, uniform=gen.WARP_UNIFORM, want_r0=True)
    heat, tally, want_r0 = CF.warp_heat(ev)
    got = {int.from_bytes(k, "little"): (int.from_bytes(v[:8], "little"), int.from_bytes(v[8:], "little"))
           for k, v in maps[0].hash_items().items()}
    assert got == heat
    assert np.array_equal(maps[1].array_u64(), tally)
    assert np.array_equal(r0, want_r0)
    assert tally[8, 0] > 0 and tally[9, 0] > 0 and (want_r0 > 0).any() and (want_r0 == 0).any()
