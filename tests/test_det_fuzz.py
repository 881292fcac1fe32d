"""Deterministic mode's claim, fuzzed on the oracle: for every program it accepts, the final
maps, the multiset of ring-buffer payloads and each event's R0 are the same whatever the
order of the events (the reading of Sec. 4.4.3's relaxed consistency).

Random programs mix ctx loads, ALU work, array and hash updates (ADD / OR / XOR / AND at
4 and 8 bytes, fetching or not, max / min helpers), loads of map values, branches, ring
output, plain stores and exchanges; the verifier refuses many.  Each accepted one runs on
the oracle over the same events in three orders.  Hash inserts use the insert idiom, whose
NULL branch leads to the same side effects either way: the one documented hole (a branch
on NULL-ness with different side effects) is left out by construction.
"""
import numpy as np
import pytest

import oracle as O
from tests.asmtext import assemble

gx = pytest.importorskip("paper_2512_12615_gb300")

SPECS = [dict(type=2, key_size=4, value_size=16, max_entries=8),
         dict(type=1, key_size=8, value_size=16, max_entries=4096),
         dict(type=27, key_size=0, value_size=0, max_entries=1 << 16)]


class Gen:
    def __init__(self, rng):
        self.rng, self.lines, self.label = rng, ["mov r6 r1", "ldx8 r7 r6 0", "ldx8 r8 r6 8"], 0
        self.insert = [int(rng.integers(0, 3)), 0]  # the program's insert constant (two on purpose, rarely)
        self.last_off = 0  # atomics reuse offsets, so that widths and operations meet on one word

    def r(self):
        return ["r7", "r8"][int(self.rng.integers(0, 2))]

    def fresh(self):
        self.label += 1
        return f"L{self.label}"

    def array_value(self, skip):
        k = self.r()
        self.lines += [f"mov r1 {k}", "and r1 7", "stx4 r10 -4 r1", "ld_map r1 0", "mov r2 r10", "add r2 -4",
                       "call map_lookup_elem", f"jeq r0 0 {skip}"]

    def hash_value(self, skip):
        k = self.r()
        have = self.fresh()
        c = self.insert[0] if self.rng.random() < 0.9 else self.insert[0] + 1
        self.lines += [f"mov r1 {k}", "and r1 15", "stx8 r10 -8 r1", "ld_map r1 1", "mov r2 r10", "add r2 -8",
                       "call map_lookup_elem", f"jne r0 0 {have}", f"st8 r10 -24 {c}", "st8 r10 -16 0",
                       "ld_map r1 1", "mov r2 r10", "add r2 -8", "mov r3 r10", "add r3 -24", "mov r4 1",
                       "call map_update_elem", "ld_map r1 1", "mov r2 r10", "add r2 -8", "call map_lookup_elem",
                       f"jeq r0 0 {skip}", f"{have}:"]

    def block(self, depth=0):
        rng = self.rng
        # load, alu, array atomic, hash atomic, max/min, read back, branch, output, store, exchange, constant
        k = int(rng.choice(11, p=np.array([2, 3, 5, 4, 2, 2, 2, 2, 0.4, 0.4, 1]) / 23.8))
        a, b = self.r(), self.r()
        if k == 0:
            self.lines.append(f"ldx8 {a} r6 {8 * int(rng.integers(0, 4))}")
        elif k == 1:
            op = ["add", "xor", "mul", "and", "or", "rsh"][int(rng.integers(0, 6))]
            self.lines.append(f"{op} {a} {b}" if op != "rsh" else f"rsh {a} {int(rng.integers(1, 9))}")
        elif k in (2, 3):  # an atomic on an array or hash value
            skip = self.fresh()
            (self.array_value if k == 2 else self.hash_value)(skip)
            size = [4, 8][int(rng.integers(0, 2))]
            op = ["add", "or", "xor", "and"][int(rng.integers(0, 4))]
            off = self.last_off & ~(size - 1) if rng.random() < 0.5 else int(rng.integers(0, 16 // size)) * size
            self.last_off = off
            fetch = "_fetch" if rng.random() < 0.15 else ""
            self.lines += [f"mov r9 {b}", f"atomic{size} {op}{fetch} r0 {off} r9"]
            if fetch and rng.random() < 0.5:
                self.lines.append(f"mov {b} r9")  # the fetched (order-dependent) value flows on
            self.lines.append(f"{skip}:")
        elif k == 4:  # max / min helper
            skip = self.fresh()
            self.array_value(skip)
            h = ["atomic_max_u64", "atomic_min_u64"][int(rng.integers(0, 2))]
            self.lines += ["mov r1 r0", f"add r1 {8 * int(rng.integers(0, 2))}", f"mov r2 {b}", f"call {h}",
                           f"{skip}:"]
        elif k == 5:  # a map value read back
            skip = self.fresh()
            self.array_value(skip)
            self.lines += [f"ldx8 {b} r0 {8 * int(rng.integers(0, 2))}"]
            if rng.random() < 0.5:  # keep it small, so that a branch on it goes both ways
                self.lines.append(f"and {b} 7")
            self.lines.append(f"{skip}:")
        elif k == 6 and depth < 2:  # a branch around a nested block
            skip = self.fresh()
            self.lines.append(f"jgt {a} {int(rng.integers(0, 8))} {skip}")
            self.block(depth + 1)
            self.lines.append(f"{skip}:")
        elif k == 7:  # ring output of a register
            self.lines += [f"stx8 r10 -40 {a}", "ld_map r1 2", "mov r2 r10", "add r2 -40", "mov r3 8", "mov r4 0",
                           "call ringbuf_output"]
        elif k == 8:  # a plain store into a map value
            skip = self.fresh()
            self.array_value(skip)
            self.lines += [f"stx8 r0 {8 * int(rng.integers(0, 2))} {b}", f"{skip}:"]
        elif k == 9:  # an exchange
            skip = self.fresh()
            self.array_value(skip)
            self.lines += [f"mov r9 {b}", "atomic8 xchg r0 0 r9", f"{skip}:"]
        else:
            self.lines.append(f"mov {a} {int(rng.integers(0, 5))}")

    def program(self):
        for _ in range(int(self.rng.integers(2, 8))):
            self.block()
        self.lines += [f"mov r0 {self.r()}" if self.rng.random() < 0.6 else "mov r0 0", "exit"]
        return self.lines


def outcome(prog, ev, order):
    maps = O.maps_from_specs(SPECS)
    r0, _ = O.run(prog, maps, ev[order], 32, want_r0=True)
    back = np.empty_like(r0)
    back[order] = r0  # R0 of each original event
    recs, dropped = maps[2].ringbuf_records()
    return (maps[0].array_values().tobytes(), sorted(maps[1].hash_items().items()),
            sorted(p for _, p in recs), dropped, back.tolist())


def test_accepted_programs_do_not_depend_on_event_order():
    rng = np.random.default_rng(20240)
    accepted = 0
    for i in range(2000):
        lines = Gen(rng).program()
        prog = assemble(lines).prog()
        if gx.verify(prog, SPECS, 32, deterministic=True)[0] != 0:
            continue
        accepted += 1
        ev = rng.integers(0, 12, size=(300, 4), dtype=np.uint64)  # small values: keys and slots collide
        ev[::7] = rng.integers(0, 2**40, size=(len(ev[::7]), 4), dtype=np.uint64)
        first = outcome(prog, ev, np.arange(len(ev)))
        for _ in range(2):
            assert outcome(prog, ev, rng.permutation(len(ev))) == first, (i, lines)
    assert accepted >= 500, accepted
