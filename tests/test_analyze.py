"""Which maps may combine their updates per thread block (host only, gx_analyze).

Block-private combining (the per-SM shards merged into the global map, Sec. 5.3) is only
invisible when the program never observes a map's values: every access must be a
non-fetching commutative update (ADD / OR / AND / XOR atomics, the atomic max / min
helpers) at a constant offset, with one operation per 4-byte word.  Each test below
changes one thing about the access and checks the outcome.
"""
import pytest

import paper_2512_12615_gb300 as gx
from tests.asmtext import assemble
from workloads import programs as P

VAL = dict(type=gx.MAP_ARRAY, key_size=4, value_size=16, max_entries=16)
HASH = dict(type=gx.MAP_HASH, key_size=8, value_size=16, max_entries=64)
RING = dict(type=gx.MAP_RINGBUF, key_size=0, value_size=0, max_entries=4096)

# r6 = ctx; r0 = &map0[3] (or skip to the end when NULL)
PRE = ["mov r6 r1", "st4 r10 -4 3", "ld_map r1 0", "mov r2 r10", "add r2 -4", "call map_lookup_elem",
       "jeq r0 0 out"]
POST = ["out:", "mov r0 0", "exit"]


def mask(body, maps=(VAL,), det=False, ctx=32):
    rc, info, log = gx.analyze(assemble(PRE + body + POST).prog(), list(maps), ctx, deterministic=det)
    assert rc == 0, log
    return info.combinable_maps


def test_atomic_add_is_combinable():
    assert mask(["mov r1 1", "atomic8 add r0 0 r1"]) == 1


@pytest.mark.parametrize("op", ["add", "or", "and", "xor"])
@pytest.mark.parametrize("size", [4, 8])
def test_each_non_fetching_atomic_is_combinable(op, size):
    assert mask(["mov r1 6", f"atomic{size} {op} r0 8 r1"]) == 1


def test_atomic_max_and_min_helpers_are_combinable():
    assert mask(["mov r1 r0", "mov r7 r0", "mov r2 9", "call atomic_max_u64",
                 "mov r1 r7", "add r1 8", "mov r2 9", "call atomic_min_u64"]) == 1


def test_different_ops_on_different_words_are_combinable():
    assert mask(["mov r1 1", "atomic8 add r0 0 r1", "atomic4 or r0 8 r1", "atomic4 xor r0 12 r1"]) == 1


def test_load_of_the_value_is_not():
    assert mask(["mov r1 1", "atomic8 add r0 0 r1", "ldx8 r1 r0 8"]) == 0


@pytest.mark.parametrize("store", ["st8 r0 0 5", "stx8 r0 0 r1"])
def test_plain_store_is_not(store):
    assert mask(["mov r1 1", store]) == 0


@pytest.mark.parametrize("kind", ["add_fetch", "or_fetch", "xchg", "cmpxchg"])
def test_fetching_or_exchanging_atomic_is_not(kind):
    # the pointer in r7: CMPXCHG takes its expected value from R0
    assert mask(["mov r7 r0", "mov r0 0", "mov r1 1", f"atomic8 {kind} r7 0 r1"]) == 0


def test_two_ops_on_one_word_is_not():
    assert mask(["mov r1 1", "atomic8 add r0 0 r1", "atomic8 or r0 0 r1"]) == 0


def test_two_widths_on_one_word_is_not():
    assert mask(["mov r1 1", "atomic8 add r0 0 r1", "atomic4 add r0 0 r1"]) == 0


def test_variable_offset_is_not():
    assert mask(["ldx4 r3 r6 24", "and r3 1", "lsh r3 3", "add r0 r3", "mov r1 1", "atomic8 add r0 0 r1"]) == 0


def test_value_handed_to_a_helper_is_not():
    # ringbuf_output reads the 16 value bytes
    body = ["mov r1 1", "atomic8 add r0 0 r1", "mov r2 r0", "ld_map r1 1", "mov r3 16", "mov r4 0",
            "call ringbuf_output"]
    assert mask(body, maps=(VAL, RING)) == 0


def test_value_as_lookup_key_is_not():
    body = ["mov r1 1", "atomic8 add r0 0 r1", "mov r2 r0", "ld_map r1 0", "call map_lookup_elem"]
    assert mask(body) == 0


def test_lookup_only_map_is_not_marked():
    assert mask(["mov r1 r0"]) == 0


HASH_PRE = ["mov r6 r1", "ldx8 r7 r6 0", "stx8 r10 -8 r7", "ld_map r1 0", "mov r2 r10", "add r2 -8",
            "call map_lookup_elem", "jne r0 0 have",
            "st8 r10 -24 0", "st8 r10 -16 0", "ld_map r1 0", "mov r2 r10", "add r2 -8", "mov r3 r10",
            "add r3 -24", "mov r4 {flags}", "call map_update_elem", "ja out",
            "have:", "mov r1 1", "atomic8 add r0 0 r1"]


def hash_mask(flags, det=False):
    prog = assemble([l.format(flags=flags) for l in HASH_PRE] + POST).prog()
    rc, info, log = gx.analyze(prog, [HASH], 32, deterministic=det)
    assert rc == 0, log
    return info.combinable_maps


def test_insert_if_absent_keeps_hash_combinable():
    assert hash_mask(1) == 1  # BPF_NOEXIST
    assert hash_mask(1, det=True) == 1


@pytest.mark.parametrize("flags", [0, 2])  # BPF_ANY, BPF_EXIST overwrite an existing value
def test_overwriting_update_is_not(flags):
    assert hash_mask(flags) == 0


def test_ring_buffer_is_never_marked():
    body = ["mov r1 1", "atomic8 add r0 0 r1", "ld_map r1 1", "mov r2 r10", "add r2 -4", "mov r3 4", "mov r4 0",
            "call ringbuf_output"]
    assert mask(body, maps=(VAL, RING)) == 1


def test_workload_programs():
    prog, maps, cs = P.counting()
    assert gx.analyze(prog, maps, cs)[1].combinable_maps == 1
    prog, maps, cs = P.page_heat()
    assert gx.analyze(prog, maps, cs)[1].combinable_maps == 3  # heat (hash) and tally (array)
    prog, maps, cs = P.latency()
    assert gx.analyze(prog, maps, cs)[1].combinable_maps == 1  # histogram; the ring buffer never


def test_rejected_program_reports_nothing():
    rc, info, log = gx.analyze(assemble(["exit"]).prog(), [], 32)
    assert rc == gx.E_VERIFY and info.combinable_maps == 0 and "R0" in log
