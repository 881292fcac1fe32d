"""Merging map copies across engines (the multi-GPU read-time merge), host only.

The reference is the sequential oracle over a whole batch.  The oracle runs over disjoint
parts of the batch, each with maps of its own and its part's global event base, stand in
for the engines of several GPUs.  Merged by `gx_merge_ops` and `merge.py`, their maps
must equal the reference's exactly, for every workload program, the all-operations
program with non-zero starting values, a non-zero insert constant and the 64 generated
programs.  The last test does the same across two gloo ranks.
"""
import os
import socket

import numpy as np
import pytest

import oracle as O
from tests.asmtext import assemble
from workloads import gen
from workloads import programs as P

gx = pytest.importorskip("paper_2512_12615_gb300")
from paper_2512_12615_gb300 import merge as M  # noqa: E402


def snapshot(m):
    if m.type == O.MAP_HASH:
        return m.hash_items()
    if m.type == O.MAP_ARRAY:
        return m.array_values()
    return m.ringbuf_records()


def run_parts(prog, specs, cs, ev, cuts, init=None):
    """The oracle over ev[cuts[j]:cuts[j+1]] with maps of its own per part: per-part snapshots."""
    raw = np.ascontiguousarray(ev).view(np.uint8).reshape(-1, cs)
    parts = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        maps = O.maps_from_specs(specs)
        for m, v in zip(maps, init or [None] * len(maps)):
            if v is not None:
                for k in range(m.max_entries):
                    m.update(int(k).to_bytes(4, "little"), v[k * m.value_size:(k + 1) * m.value_size])
        O.run(prog, maps, raw[a:b], cs, event_idx_base=a)
        parts.append([snapshot(m) for m in maps])
    return parts


def merge_parts(prog, specs, cs, parts, init=None):
    start = None if not init else [None if v is None else np.frombuffer(v, np.uint8) for v in init]
    return M.merge_snapshots(prog, specs, cs, parts, init=start)


def assert_merge_equals_whole(prog, specs, cs, ev, cuts, init=None):
    whole = run_parts(prog, specs, cs, ev, [0, cuts[-1]], init)[0]
    merged = merge_parts(prog, specs, cs, run_parts(prog, specs, cs, ev, cuts, init), init)
    for s, w, m in zip(specs, whole, merged):
        if s["type"] == O.MAP_ARRAY:
            assert np.array_equal(w, m)
        else:
            assert w == m


def cuts_for(n, k, seed):
    inner = np.sort(np.random.default_rng(seed).choice(np.arange(1, n), size=k - 1, replace=False))
    return [0] + [int(c) for c in inner] + [n]


@pytest.mark.parametrize("k", [2, 3, 5])
@pytest.mark.parametrize("name", ["counting", "page_heat", "latency"])
def test_workload_copies_merge_exactly(name, k):
    if name == "counting":
        (prog, specs, cs), ev = P.counting(), gen.uniform_events(20_011, seed=1)
    elif name == "page_heat":
        (prog, specs, cs), ev = P.page_heat(), gen.pageheat_events(40_009, seed=2)
        ev["size"][::97] = 3
        ev["addr"][7::89] |= np.uint64(1)
    else:
        (prog, specs, cs), ev = P.latency(ring_bytes=1 << 22), gen.latency_pairs(20_003, seed=3)
    n = len(np.ascontiguousarray(ev).view(np.uint8)) // cs
    assert_merge_equals_whole(prog, specs, cs, ev, cuts_for(n, k, seed=k))


def test_every_operation_with_starting_values():
    """ADD (4 and 8 bytes, near the wrap), OR, AND and MIN over non-zero starting values, XOR,
    MAX, 4-byte OR / XOR, in an array map and in a hash map; 4 uneven parts."""
    from tests.test_gpu_shards import ALLOPS, SPECS, allops_events, allops_init

    prog = assemble(ALLOPS).prog()
    assert_merge_equals_whole(prog, SPECS, 32, allops_events(30_001, seed=4), cuts_for(30_001, 4, seed=9),
                              init=allops_init())


def test_nonzero_insert_constant():
    """Keys inserted as {5, 2^64 - 16} then added to and xor-ed: a key held by several copies
    starts from the insert constant, not from zero."""
    lines = ["ldx8 r7 r1 0", "ldx8 r8 r1 8", "and r7 15", "stx8 r10 -8 r7", "ld_map r1 0", "mov r2 r10", "add r2 -8",
             "call map_lookup_elem", "jne r0 0 have", "st8 r10 -24 5", "st8 r10 -16 -16", "ld_map r1 0", "mov r2 r10",
             "add r2 -8", "mov r3 r10", "add r3 -24", "mov r4 1", "call map_update_elem", "ld_map r1 0", "mov r2 r10",
             "add r2 -8", "call map_lookup_elem", "jeq r0 0 out", "have:", "atomic8 add r0 0 r8",
             "atomic8 xor r0 8 r8", "out:", "mov r0 0", "exit"]
    specs = [dict(type=1, key_size=8, value_size=16, max_entries=64)]
    prog = assemble(lines).prog()
    rc, ops, insert, _ = gx.merge_ops(prog, specs, 16, 0)
    assert rc == 0 and list(ops) == [0x11, 0x11, 0x04, 0x04]  # the XOR merges per 4-byte word
    assert insert == (5).to_bytes(8, "little") + (2**64 - 16).to_bytes(8, "little")
    ev = np.random.default_rng(5).integers(0, 2**63, size=(5_000, 2), dtype=np.uint64)
    assert_merge_equals_whole(prog, specs, 16, ev, [0, 1_000, 2_500, 5_000])


@pytest.mark.parametrize("p", range(64))
def test_generated_programs_merge_exactly(p):
    prog, specs, cs = P.batch_programs()[p]
    ev = gen.uniform_events(3_001, seed=600 + p)
    assert_merge_equals_whole(prog, specs, cs, ev, cuts_for(3_001, 3, seed=p))


def test_ring_records_come_back_in_event_order():
    """An engine's drained ring holds its records in reservation order, and copies may arrive
    in any order: the merge orders them by event index, each event's records kept in
    emission order.  Two records per event, so that order is visible."""
    lines = ["ldx8 r6 r1 0", "ld_map r1 0", "mov r2 8", "mov r3 0", "call ringbuf_reserve", "jeq r0 0 out",
             "stx8 r0 0 r6", "mov r1 r0", "mov r2 0", "call ringbuf_submit", "ld_map r1 0", "mov r2 8", "mov r3 0",
             "call ringbuf_reserve", "jeq r0 0 out", "add r6 1", "stx8 r0 0 r6", "mov r1 r0", "mov r2 0",
             "call ringbuf_submit", "out:", "mov r0 0", "exit"]
    specs = [dict(type=27, key_size=0, value_size=0, max_entries=1 << 16)]
    prog = assemble(lines).prog()
    ev = np.arange(600, dtype=np.uint64).reshape(300, 2) * np.uint64(10)
    whole = run_parts(prog, specs, 16, ev, [0, 300])[0][0]
    rng = np.random.default_rng(6)
    copies = []
    for part in run_parts(prog, specs, 16, ev, [0, 90, 200, 300]):
        recs, dropped = part[0]
        events = sorted({i for i, _ in recs})
        rng.shuffle(events)  # reservation order: events interleaved, each event's records in order
        copies.append(([r for e in events for r in recs if r[0] == e], dropped))
    assert M.merge_ring(copies[::-1]) == whole and len(whole[0]) == 600


def test_merge_codes_and_refusals():
    prog, specs, cs = P.page_heat()
    rc, ops, insert, _ = gx.merge_ops(prog, specs, cs, 0)
    assert rc == 0 and list(ops) == [gx.MERGE_W8 | gx.MERGE_ADD] * 2 + [gx.MERGE_W8 | gx.MERGE_MAX] * 2
    assert insert == bytes(16)
    assert gx.merge_ops(prog, specs, cs, 1)[2] is None  # the tally is never inserted into
    # a word added at two widths is order-dependent: refused by deterministic verification
    arr = [dict(type=2, key_size=4, value_size=8, max_entries=1)]
    look = ["st4 r10 -4 0", "ld_map r1 0", "mov r2 r10", "add r2 -4", "call map_lookup_elem", "jeq r0 0 out",
            "mov r1 1"]
    rc, _, _, log = gx.merge_ops(assemble(look + ["atomic8 add r0 0 r1", "atomic4 add r0 0 r1", "out:", "mov r0 0",
                                                  "exit"]).prog(), arr, 16, 0)
    assert rc == gx.E_VERIFY and "two widths" in log
    # bitwise operations at two widths merge per 4-byte word
    rc, ops, _, log = gx.merge_ops(assemble(look + ["atomic8 or r0 0 r1", "atomic4 or r0 0 r1", "out:", "mov r0 0",
                                                    "exit"]).prog(), arr, 16, 0)
    assert rc == 0 and list(ops) == [gx.MERGE_OR, gx.MERGE_OR], log
    # inserts of two different constants: the first event's stay, so the order decides
    hs = [dict(type=1, key_size=8, value_size=8, max_entries=4)]
    ins = ["st8 r10 -8 1", "st8 r10 -16 {}", "ld_map r1 0", "mov r2 r10", "add r2 -8", "mov r3 r10", "add r3 -16",
           "mov r4 1", "call map_update_elem"]
    two = [x.format(0) for x in ins] + [x.format(1) for x in ins] + ["mov r0 0", "exit"]
    rc, _, _, log = gx.merge_ops(assemble(two).prog(), hs, 16, 0)
    assert rc == gx.E_VERIFY and "different constants" in log  # order-dependent: refused by the verifier
    # a plain store into map memory is refused in deterministic mode
    rc, _, _, _ = gx.merge_ops(assemble(look + ["stx8 r0 0 r1", "out:", "mov r0 0", "exit"]).prog(), arr, 16, 0)
    assert rc == gx.E_VERIFY
    # copies that differ where no update reaches are not merged silently
    with pytest.raises(ValueError):
        M.merge_array([0, 0], [np.zeros((1, 8), np.uint8), np.ones((1, 8), np.uint8)])


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out) -> None:
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ok = []
        for build, ev in ((P.page_heat, gen.pageheat_events(30_000, seed=8)),
                          (lambda: P.latency(ring_bytes=1 << 22), gen.latency_pairs(10_000, seed=9))):
            prog, specs, cs = build()
            n = len(np.ascontiguousarray(ev).view(np.uint8)) // cs
            cuts = [n * r // world for r in range(world + 1)]
            mine = run_parts(prog, specs, cs, ev, cuts[rank:rank + 2])[0]  # this rank's part only
            merged = M.merge_across_ranks(dist, prog, specs, cs, mine)
            whole = run_parts(prog, specs, cs, ev, [0, n])[0]
            ok.append(all(np.array_equal(w, m) if s["type"] == O.MAP_ARRAY else w == m
                          for s, w, m in zip(specs, whole, merged)))
        out.put((rank, ok))
    finally:
        dist.destroy_process_group()


def test_two_ranks_merge_their_maps():
    """Two gloo ranks, each with half of a batch and maps of its own, gather and merge their
    snapshots: both end with the maps of the whole batch (page-heat; latency with its ring)."""
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, [True, True]), (1, [True, True])]
