"""Verifier invariants (host only, through the C ABI's gx_verify).

Accepts every workload program; rejects each class of unsafe program the paper's
verification has to exclude (Sec. 4.4: bounded loops, memory safety, typed access) and,
in deterministic mode, programs whose results could depend on event order.
"""
import json
import os

import numpy as np
import pytest

import paper_2512_12615_gb300 as gx
from tests.asmtext import assemble
from workloads import programs as P
from workloads.asm import Asm

ARRAY = dict(type=gx.MAP_ARRAY, key_size=4, value_size=8, max_entries=16)
HASH = dict(type=gx.MAP_HASH, key_size=8, value_size=16, max_entries=64)
RING = dict(type=gx.MAP_RINGBUF, key_size=0, value_size=0, max_entries=4096)


def ok(lines, maps=(), ctx=32, det=False):
    rc, log = gx.verify(assemble(lines).prog(), list(maps), ctx, deterministic=det)
    assert rc == 0, log


def rejected(lines, maps=(), ctx=32, det=False, why=""):
    rc, log = gx.verify(assemble(lines).prog() if isinstance(lines, list) else lines, list(maps), ctx,
                        deterministic=det)
    assert rc == gx.E_VERIFY, f"accepted; expected rejection ({why})"
    if why:
        assert why in log, log
    return log


@pytest.mark.parametrize("build", [P.counting, P.page_heat, P.latency])
@pytest.mark.parametrize("det", [False, True])
def test_accepts_workload_programs(build, det):
    prog, maps, cs = build()
    rc, log = gx.verify(prog, maps, cs, deterministic=det)
    assert rc == 0, log


def test_accepts_random_batch_programs_deterministic():
    for i, (prog, maps, cs) in enumerate(P.batch_programs()):
        rc, log = gx.verify(prog, maps, cs, deterministic=True)
        assert rc == 0, (i, log)


def test_accepts_handworked_programs():
    cases = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "handworked.json")))["cases"]
    for c in cases:
        maps = [dict(m) for m in c.get("maps", [])]
        for m in maps:
            if m["type"] == gx.MAP_RINGBUF:
                m["max_entries"] = max(m["max_entries"], 4096)
        ev = np.array(c["events"])
        rc, log = gx.verify(assemble(c["asm"]).prog(), maps, 8 * ev.shape[1])
        assert rc == 0, (c["name"], log)


# ---------------------------------------------------------------- control flow
def test_rejects_infinite_self_jump():
    rejected(["mov r0 0", "l:", "ja l"], why="infinite loop")


def test_rejects_unbounded_counter_loop():
    rejected(["mov r0 0", "l:", "add r0 1", "ja l"], why="too complex")


def test_rejects_data_dependent_unbounded_loop():
    rejected(["ldx8 r2 r1 0", "mov r0 0", "l:", "add r0 1", "jne r0 r2 l", "exit"], why="too complex")


def test_accepts_constant_bound_loop():
    ok(["mov r0 0", "mov r2 0", "l:", "add r0 r2", "add r2 1", "jlt r2 100 l", "exit"])


def test_rejects_jump_out_of_range():
    rejected(Asm().raw(0x05, 0, 0, 5, 0).mov("r0", 0).exit().prog(), [], 32, why="jump out of range")


def test_rejects_fall_off_end():
    rejected(["mov r0 0"], why="falls off the end")


def test_rejects_jump_into_ld_imm64():
    prog = Asm().raw(0x05, 0, 0, 1, 0).ld_imm64("r0", 5).exit().prog()
    rejected(prog, [], 32, why="middle of a 64-bit immediate")


# ---------------------------------------------------------------- registers
def test_rejects_uninitialised_read():
    rejected(["mov r0 r3", "exit"], why="uninitialised R3")


def test_rejects_uninitialised_r0_at_exit():
    rejected(["exit"], why="uninitialised R0")


def test_rejects_write_to_r10():
    rejected(["mov r10 0", "mov r0 0", "exit"], why="R10 is read-only")


def test_rejects_clobbered_argument_register_after_call():
    rejected(["st4 r10 -4 0", "ld_map r1 0", "mov r2 r10", "add r2 -4", "call map_lookup_elem", "mov r0 r2", "exit"],
             [ARRAY], why="uninitialised R2")


def test_rejects_pointer_returned():
    rejected(["mov r0 r10", "exit"], why="not a scalar")


def test_rejects_pointer_arithmetic_other_than_add():
    rejected(["mov r2 r10", "mul r2 2", "mov r0 0", "exit"], why="arithmetic on a pointer")


def test_rejects_32bit_copy_of_pointer():
    rejected(["mov32 r2 r10", "mov r0 0", "exit"], why="32-bit move of a pointer")


# ---------------------------------------------------------------- memory
def test_rejects_stack_below_512():
    rejected(["st8 r10 -520 0", "mov r0 0", "exit"], why="stack access out of bounds")


def test_rejects_stack_at_frame_pointer():
    rejected(["stx8 r10 0 r1", "mov r0 0", "exit"], why="stack access out of bounds")


def test_rejects_uninitialised_stack_read():
    rejected(["ldx8 r0 r10 -8", "exit"], why="uninitialised stack")


def test_rejects_misaligned_stack_access():
    rejected(["st8 r10 -12 0", "mov r0 0", "exit"], why="misaligned")


def test_rejects_ctx_out_of_bounds_and_write():
    rejected(["ldx8 r0 r1 32", "exit"], why="ctx read out of bounds")
    rejected(["st4 r1 0 1", "mov r0 0", "exit"], why="read-only")


LOOKUP = ["st4 r10 -4 0", "ld_map r1 0", "mov r2 r10", "add r2 -4", "call map_lookup_elem"]


def test_rejects_unchecked_lookup_result():
    rejected(LOOKUP + ["ldx8 r0 r0 0", "exit"], [ARRAY], why="load through a map_value_or_null")


def test_rejects_map_value_out_of_bounds():
    rejected(LOOKUP + ["jeq r0 0 out", "ldx8 r0 r0 8", "exit", "out:", "mov r0 0", "exit"], [ARRAY],
             why="out of bounds")
    ok(LOOKUP + ["jeq r0 0 out", "ldx8 r0 r0 0", "exit", "out:", "mov r0 0", "exit"], [ARRAY])


def test_rejects_variable_offset_beyond_value():
    prog = ["mov r6 r1"] + LOOKUP + ["jeq r0 0 out", "ldx8 r3 r6 0", "and r3 1", "lsh r3 3", "add r0 r3",
                                     "ldx8 r0 r0 0", "exit", "out:", "mov r0 0", "exit"]
    rejected(prog, [ARRAY], why="out of bounds")
    ok(prog, [dict(ARRAY, value_size=16)])


def test_rejects_pointer_stored_into_map():
    rejected(LOOKUP + ["jeq r0 0 out", "stx8 r0 0 r10", "out:", "mov r0 0", "exit"], [ARRAY], why="pointer stored")


def test_rejects_key_with_uninitialised_bytes():
    rejected(["ld_map r1 0", "mov r2 r10", "add r2 -8", "call map_lookup_elem", "mov r0 0", "exit"], [HASH],
             why="uninitialised stack byte")


def test_rejects_unknown_helper_and_legacy_packet_loads():
    rejected(["call 9999", "mov r0 0", "exit"], why="unknown helper")
    rejected(Asm().raw(0x20, 0, 0, 0, 0).exit().prog(), [], 32, why="legacy packet access")
    rejected(Asm().raw(0x40, 0, 1, 0, 0).exit().prog(), [], 32, why="legacy packet access")


def test_rejects_bad_map_index():
    rejected(["ld_map r1 3", "mov r0 0", "exit"], [ARRAY], why="map index")


# ---------------------------------------------------------------- ring buffer
RESERVE = ["ld_map r1 0", "mov r2 48", "mov r3 0", "call ringbuf_reserve"]


def test_rejects_leaked_reservation():
    rejected(RESERVE + ["mov r0 0", "exit"], [RING], why="neither submitted nor discarded")
    rejected(RESERVE + ["jeq r0 0 out", "mov r0 0", "exit", "out:", "exit"], [RING],
             why="neither submitted nor discarded")


def test_accepts_reserve_submit_and_rejects_use_after_submit():
    good = RESERVE + ["jeq r0 0 out", "mov r6 r0", "st8 r6 40 7", "mov r1 r6", "mov r2 0", "call ringbuf_submit",
                      "out:", "mov r0 0", "exit"]
    ok(good, [RING])
    bad = RESERVE + ["jeq r0 0 out", "mov r6 r0", "mov r1 r6", "mov r2 0", "call ringbuf_submit", "st8 r6 0 1",
                     "out:", "mov r0 0", "exit"]
    rejected(bad, [RING], why="uninitialised R6")


def test_rejects_reservation_write_out_of_bounds():
    rejected(RESERVE + ["jeq r0 0 out", "st8 r0 48 1", "mov r1 r0", "mov r2 0", "call ringbuf_submit", "out:",
                        "mov r0 0", "exit"], [RING], why="out of bounds")


# ---------------------------------------------------------------- deterministic mode
VALUE = LOOKUP + ["jeq r0 0 out"]


def test_det_rejects_branch_on_map_value():
    prog = VALUE + ["ldx8 r3 r0 0", "jeq r3 5 out", "mov r0 1", "exit", "out:", "mov r0 0", "exit"]
    ok(prog, [ARRAY])
    rejected(prog, [ARRAY], det=True, why="order-dependent")


def test_det_rejects_map_value_in_r0_and_plain_stores():
    rejected(VALUE + ["ldx8 r0 r0 0", "exit", "out:", "mov r0 0", "exit"], [ARRAY], det=True, why="R0")
    rejected(VALUE + ["st8 r0 0 1", "out:", "mov r0 0", "exit"], [ARRAY], det=True, why="plain store")


def test_det_rejects_exchange_and_fetch_result_use():
    rejected(VALUE + ["mov r3 1", "atomic8 xchg r0 0 r3", "out:", "mov r0 0", "exit"], [ARRAY], det=True,
             why="exchange")
    rejected(VALUE + ["mov r3 1", "atomic8 add_fetch r0 0 r3", "mov r0 r3", "exit", "out:", "mov r0 0", "exit"],
             [ARRAY], det=True, why="R0")
    ok(VALUE + ["mov r3 1", "atomic8 add r0 0 r3", "out:", "mov r0 0", "exit"], [ARRAY], det=True)


def test_det_rejects_non_insert_updates_and_deletes():
    upd = ["st8 r10 -8 1", "st8 r10 -24 0", "st8 r10 -16 0", "ld_map r1 0", "mov r2 r10", "add r2 -8", "mov r3 r10",
           "add r3 -24"]
    ok(upd + ["mov r4 1", "call map_update_elem", "mov r0 0", "exit"], [HASH], det=True)
    rejected(upd + ["mov r4 0", "call map_update_elem", "mov r0 0", "exit"], [HASH], det=True, why="NOEXIST")
    rejected(["st8 r10 -8 1", "ld_map r1 0", "mov r2 r10", "add r2 -8", "call map_delete_elem", "mov r0 0", "exit"],
             [HASH], det=True, why="delete")


def test_det_rejects_variable_insert_value():
    prog = ["st8 r10 -8 1", "ldx8 r3 r1 0", "stx8 r10 -24 r3", "st8 r10 -16 0", "ld_map r1 0", "mov r2 r10",
            "add r2 -8", "mov r3 r10", "add r3 -24", "mov r4 1", "call map_update_elem", "mov r0 0", "exit"]
    ok(prog, [HASH])
    rejected(prog, [HASH], det=True, why="constant bytes")


def test_det_rejects_update_status_in_branch():
    prog = ["st8 r10 -8 1", "st8 r10 -24 0", "st8 r10 -16 0", "ld_map r1 0", "mov r2 r10", "add r2 -8", "mov r3 r10",
            "add r3 -24", "mov r4 1", "call map_update_elem", "jeq r0 0 out", "mov r0 1", "exit", "out:", "mov r0 0",
            "exit"]
    ok(prog, [HASH])
    rejected(prog, [HASH], det=True, why="order-dependent")


def test_rejects_bad_specs_and_sizes():
    assert gx.verify(assemble(["mov r0 0", "exit"]).prog(), [], 12)[0] == gx.E_VERIFY  # ctx not a multiple of 8
    assert gx.verify(assemble(["mov r0 0", "exit"]).prog(), [dict(ARRAY, key_size=8)], 32)[0] == gx.EINVAL
    assert gx.verify(assemble(["mov r0 0", "exit"]).prog(), [dict(RING, max_entries=5000)], 32)[0] == gx.EINVAL
    big = Asm()
    for _ in range(4100):
        big.mov("r0", 0)
    big.exit()
    assert gx.verify(big.prog(), [], 32)[0] == gx.E_VERIFY


def test_det_rejects_mixed_atomic_operations_on_the_same_bytes():
    """add and xor each commute with themselves, not with each other."""
    mixed = VALUE + ["mov r3 1", "atomic8 add r0 0 r3", "atomic8 xor r0 0 r3", "out:", "mov r0 0", "exit"]
    ok(mixed, [ARRAY])
    rejected(mixed, [ARRAY], det=True, why="two different atomic operations")
    split = VALUE + ["mov r3 1", "atomic8 add r0 0 r3", "mov r1 r0", "add r1 8", "mov r2 5",
                     "call atomic_max_u64", "out:", "mov r0 0", "exit"]
    ok(split, [dict(ARRAY, value_size=16)], det=True)
    rejected(split, [ARRAY], det=True, why="out of bounds")
    same_word = VALUE + ["mov r3 1", "atomic8 add r0 0 r3", "mov r1 r0", "mov r2 5", "call atomic_max_u64",
                         "out:", "mov r0 0", "exit"]
    rejected(same_word, [ARRAY], det=True, why="two different atomic operations")


# ---------------------------------------------------------------- insert-only hash maps
DEL = ["mov r6 r1", "ldx8 r7 r6 0", "stx8 r10 -8 r7", "ld_map r1 0", "mov r2 r10", "add r2 -8",
       "call map_delete_elem", "mov r0 0", "exit"]


def test_delete_allowed_on_an_ordinary_hash_map():
    ok(DEL, [HASH])


def test_rejects_delete_on_an_insert_only_hash_map():
    rejected(DEL, [dict(HASH, flags=gx.MAP_F_NO_DELETE)], why="created without deletes")


@pytest.mark.parametrize("spec", [dict(ARRAY, flags=gx.MAP_F_NO_DELETE), dict(HASH, flags=2), dict(RING, flags=1)])
def test_rejects_bad_map_flags(spec):
    rc, log = gx.verify(assemble(["mov r0 0", "exit"]).prog(), [spec], 32)
    assert rc == gx.EINVAL and "invalid map spec" in log


def test_det_rejects_adds_at_two_widths():
    """A 32-bit add drops the carry a 64-bit add keeps.  On one word, two events in the two
    orders leave different values (the oracle shows it), so deterministic mode refuses
    adds to the same bytes at two widths; bitwise operations at two widths commute."""
    import oracle as O

    body = ["ldx8 r3 r6 0", "jeq r3 0 wide", "mov r3 1", "atomic4 add r7 0 r3", "ja out", "wide:", "mov r3 1",
            "atomic8 add r7 0 r3"]
    lines = ["mov r6 r1"] + VALUE + ["mov r7 r0"] + body + ["out:", "mov r0 0", "exit"]
    ok(lines, [ARRAY])
    rejected(lines, [ARRAY], det=True, why="two widths")
    ok(["mov r6 r1"] + VALUE + ["mov r7 r0"] + [b.replace("add", "or") for b in body] + ["out:", "mov r0 0", "exit"],
       [ARRAY], det=True)
    ok(VALUE + ["mov r3 1", "atomic8 add r0 0 r3", "atomic4 add r0 8 r3", "out:", "mov r0 0", "exit"],
       [dict(ARRAY, value_size=16)], det=True)  # disjoint words
    # the word starts at 2^32 - 1: add32 then add64 gives 1, add64 then add32 gives 2^32 + 1
    prog = assemble(lines).prog()
    finals = []
    for order in ([1, 0], [0, 1]):
        maps = O.maps_from_specs([ARRAY])
        maps[0].update((0).to_bytes(4, "little"), (2**32 - 1).to_bytes(8, "little"))  # the key LOOKUP uses
        O.run(prog, maps, np.array([[order[0], 0], [order[1], 0]], dtype=np.uint64), 16)
        finals.append(int(maps[0].array_u64()[0, 0]))
    assert finals == [1, 2**32 + 1]


def test_det_rejects_inserts_of_different_constants():
    """Two events inserting one key with NOEXIST: the first one's bytes stay, so two
    different inserted constants make the result order-dependent."""
    ins = ["st8 r10 -8 1", "st8 r10 -16 {}", "ld_map r1 0", "mov r2 r10", "add r2 -8", "mov r3 r10", "add r3 -16",
           "mov r4 1", "call map_update_elem"]
    hs = [dict(HASH, value_size=8)]
    same = [x.format(7) for x in ins] * 2 + ["mov r0 0", "exit"]
    two = [x.format(0) for x in ins] + [x.format(7) for x in ins] + ["mov r0 0", "exit"]
    ok(same, hs, det=True)
    ok(two, hs)
    rejected(two, hs, det=True, why="different constants")
