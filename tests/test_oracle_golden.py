"""Pins the oracle on hand-worked programs (tests/golden/handworked.json).

Each case states the rule it follows (RFC 9669 section or the Linux helper contract) and
derives the expected values by hand; the oracle must reproduce them exactly.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from tests.asmtext import assemble

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "handworked.json")
CASES = json.load(open(GOLDEN))["cases"]


def events_of(case) -> tuple:
    ev = np.array(case["events"], dtype=np.uint64)
    return ev, 8 * ev.shape[1]


def u64_pairs(items: dict):
    out = []
    for k, v in items.items():
        out.append([int.from_bytes(k, "little"), int.from_bytes(v, "little")])
    return sorted(out)


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_handworked(case):
    prog = assemble(case["asm"]).prog()
    maps = O.maps_from_specs(case.get("maps", []))
    ev, ctx_size = events_of(case)
    r0, count = O.run(prog, maps, ev, ctx_size, want_r0=True)
    exp = case["expect"]
    assert [int(x) for x in r0] == exp["r0"]
    for idx, words in exp.get("array_u64", {}).items():
        assert maps[int(idx)].array_u64()[:, 0].tolist() == words
    for idx, pairs in exp.get("hash_u64", {}).items():
        assert u64_pairs(maps[int(idx)].hash_items()) == pairs
    for idx, recs in exp.get("ring", {}).items():
        got, dropped = maps[int(idx)].ringbuf_records()
        assert [(i, p.hex()) for i, p in got] == [(i, h) for i, h in recs]
        assert dropped == exp["dropped"][idx]
    assert count > 0


def test_faults_are_reported_not_crashing():
    """Unverified programs that leave their regions stop with an error code."""
    ev = np.zeros((1, 2), dtype=np.uint64)
    # store into the read-only ctx
    with pytest.raises(O.OracleError) as e:
        O.run(assemble(["stx8 r1 0 r1", "exit"]).prog(), [], ev, 16)
    assert e.value.rc == O.EFAULT
    # read below the 512-byte stack
    with pytest.raises(O.OracleError) as e:
        O.run(assemble(["ldx8 r0 r10 -520", "exit"]).prog(), [], ev, 16)
    assert e.value.rc == O.EFAULT
    # fall off the end
    with pytest.raises(O.OracleError) as e:
        O.run(assemble(["mov r0 0"]).prog(), [], ev, 16)
    assert e.value.rc == O.EFAULT
    # endless loop hits the per-event budget
    with pytest.raises(O.OracleError) as e:
        O.run(assemble(["l:", "ja l"]).prog(), [], ev, 16, budget=1000)
    assert e.value.rc == O.EBUDGET
    # legacy packet loads are not part of the subset
    from workloads.asm import Asm
    with pytest.raises(O.OracleError) as e:
        O.run(Asm().raw(0x20, 0, 0, 0, 0).exit().prog(), [], ev, 16)
    assert e.value.rc == O.EINVAL


def test_insn_count_is_exact():
    """A straight-line program executes every slot once; LD_IMM64 counts as one."""
    prog = assemble(["ld_imm64 r0 5", "add r0 1", "exit"]).prog()
    _, count = O.run(prog, [], np.zeros((7, 2), dtype=np.uint64), 16)
    assert count == 7 * 3
    # the 10-trip loop: 2 setup + 10 * 3 + exit
    prog = assemble(["mov r0 0", "mov r2 1", "l:", "add r0 r2", "add r2 1", "jle r2 10 l", "exit"]).prog()
    _, count = O.run(prog, [], np.zeros((1, 2), dtype=np.uint64), 16)
    assert count == 2 + 30 + 1


@pytest.mark.parametrize("lines,misaligned", [
    (["st8 r10 -8 0", "ldx4 r0 r10 -6", "exit"], True),
    (["st8 r10 -8 0", "ldx4 r0 r10 -4", "exit"], False),
    (["st8 r10 -8 0", "st2 r10 -7 1", "mov r0 0", "exit"], True),
    (["st8 r10 -8 0", "mov r1 1", "atomic4 add r10 -6 r1", "mov r0 0", "exit"], True),
    (["ldx2 r0 r1 3", "exit"], True),
    (["ldx1 r0 r1 3", "exit"], False),
])
def test_strict_alignment(lines, misaligned):
    """OR_STRICT_ALIGN: an access whose address is not a multiple of its size faults (the
    engine's reading that device accesses are naturally aligned); by default alignment is free."""
    ev = np.zeros((1, 2), dtype=np.uint64)
    prog = assemble(lines).prog()
    O.run(prog, [], ev, 16)
    if misaligned:
        with pytest.raises(O.OracleError) as e:
            O.run(prog, [], ev, 16, strict_align=True)
        assert e.value.rc == O.EFAULT
    else:
        O.run(prog, [], ev, 16, strict_align=True)


def test_strict_alignment_of_the_max_helper():
    specs = [dict(type=2, key_size=4, value_size=16, max_entries=1)]
    look = ["st4 r10 -4 0", "ld_map r1 0", "mov r2 r10", "add r2 -4", "call map_lookup_elem", "jeq r0 0 out",
            "mov r1 r0", "add r1 {}", "mov r2 5", "call atomic_max_u64", "out:", "mov r0 0", "exit"]
    ev = np.zeros((1, 2), dtype=np.uint64)
    O.run(assemble([x.format(8) for x in look]).prog(), O.maps_from_specs(specs), ev, 16, strict_align=True)
    with pytest.raises(O.OracleError) as e:
        O.run(assemble([x.format(4) for x in look]).prog(), O.maps_from_specs(specs), ev, 16, strict_align=True)
    assert e.value.rc == O.EFAULT


def test_most_counts_per_event():
    """`most`: the largest instruction, helper-call and memory-operation counts of one event.
    Event 0 (word 0 = 0) takes the short path: mov, ldx, jeq, mov, exit = 5 instructions,
    1 memory operation.  Event 1 takes the long one: mov, ldx, jeq, st, ldx, ld_map (one
    instruction), mov, add, call, mov, exit = 11 instructions, 3 memory operations, 1 call."""
    lines = ["mov r6 r1", "ldx8 r2 r6 0", "jeq r2 0 out", "st4 r10 -4 0", "ldx4 r3 r10 -4", "ld_map r1 0",
             "mov r2 r10", "add r2 -4", "call map_lookup_elem", "out:", "mov r0 0", "exit"]
    specs = [dict(type=2, key_size=4, value_size=8, max_entries=1)]
    prog = assemble(lines).prog()
    for ev, want in ((np.array([[0, 0]], np.uint64), [5, 0, 1]),
                     (np.array([[0, 0], [1, 0], [0, 0]], np.uint64), [11, 1, 3])):
        most = []
        O.run(prog, O.maps_from_specs(specs), ev, 16, most=most)
        assert most == want
