"""The verifier's memory-safety proof, fuzzed on the oracle.

The engine runs verified programs without run-time bounds checks, so the proof is what
keeps device memory safe (Sec. 4.4: memory safety, bounded loops, typed access).  The
oracle checks every access against the regions an event may touch (its ctx read-only,
its stack, looked-up values, its ring reservations), and in strict-alignment mode that
every load, store and atomic is naturally aligned, and stops with EFAULT or EINVAL
otherwise, or with EBUDGET after 2^20 steps of one event.  So: every random program the
verifier accepts (loops only when their exploration ends) must run through the oracle
without any of them, over random events.

Programs mix ctx, stack and map-value accesses of every size at random offsets (in and
out of bounds, aligned or not), variable offsets with and without range checks, missing
NULL checks, helper arguments read from map values, ring reservations written at random
offsets and submitted, discarded or leaked, uninitialised stack reads and bounded loops.
"""
import numpy as np
import pytest

import oracle as O
from tests.asmtext import assemble

gx = pytest.importorskip("paper_2512_12615_gb300")

CTX = 32
SPECS = [dict(type=2, key_size=4, value_size=24, max_entries=4),
         dict(type=1, key_size=8, value_size=16, max_entries=64),
         dict(type=27, key_size=0, value_size=0, max_entries=4096)]
SIZES = [1, 2, 4, 8]


class Gen:
    def __init__(self, rng):
        self.rng, self.n = rng, 0
        self.lines = ["mov r6 r1", "ldx8 r7 r6 0", "ldx8 r8 r6 8"] + [f"st8 r10 {-8 * j} 0" for j in range(1, 9)]

    def i(self, lo, hi):
        return int(self.rng.integers(lo, hi))

    def lab(self):
        self.n += 1
        return f"L{self.n}"

    def size(self):
        return SIZES[self.i(0, 4)]

    def off(self, limit, size):
        """mostly in bounds and aligned, sometimes not"""
        r = self.rng.random()
        if r < 0.7:
            return self.i(0, max(1, limit // size)) * size
        if r < 0.85:
            return self.i(-8, limit + 8)
        return limit - size + self.i(1, 9)

    def scalar(self):
        return ["r7", "r8"][self.i(0, 2)]

    def variable_offset(self, ptr, limit):
        """ptr += a ctx-derived scalar, masked and optionally range-checked"""
        s = self.scalar()
        mask = [7, 15, 31, 255, 0xFFFF][self.i(0, 5)]
        self.lines += ["mov r4 " + s, f"and r4 {mask}"]
        if self.rng.random() < 0.5:
            self.lines.append(f"lsh r4 {self.i(0, 4)}")
        if self.rng.random() < 0.6:
            skip = self.lab()
            self.lines.append(f"jgt r4 {self.i(0, limit + 4)} {skip}")
            self.lines += [f"add {ptr} r4"]
            return skip
        self.lines.append(f"add {ptr} r4")
        return None

    def block(self):
        # ctx, stack, array value, hash value, reservation, output, loop, variable stack offset, alu
        k = int(self.rng.choice(9, p=np.array([2, 2, 3, 3, 2, 1, 1, 0.2, 1]) / 15.2))
        sz = self.size()
        if k == 0:  # ctx access
            self.lines.append(f"ldx{sz} r{self.i(7, 9)} r6 {self.off(CTX, sz)}")
            if self.rng.random() < 0.05:
                self.lines.append(f"stx{sz} r6 0 r7")
        elif k == 1:  # stack store / load
            o = -self.off(64, sz) - sz
            self.lines.append(f"stx{sz} r10 {o} r7" if self.rng.random() < 0.5 else f"st{sz} r10 {o} {self.i(0, 9)}")
            if self.rng.random() < 0.5:
                self.lines.append(f"ldx{sz} r8 r10 {-self.off(64, sz) - sz}")
        elif k in (2, 3):  # map value access through a lookup
            m = 0 if k == 2 else 1
            vs = SPECS[m]["value_size"]
            out = self.lab()
            key = "stx4 r10 -4 r9" if m == 0 else "stx8 r10 -16 r9"
            self.lines += [f"mov r9 {self.scalar()}", f"and r9 {[3, 7][self.i(0, 2)]}", key, f"ld_map r1 {m}",
                           "mov r2 r10", f"add r2 {-4 if m == 0 else -16}", "call map_lookup_elem"]
            if self.rng.random() < 0.9:
                self.lines.append(f"jeq r0 0 {out}")
            skip = self.variable_offset("r0", vs) if self.rng.random() < 0.3 else None
            o = self.off(vs, sz)
            r = self.rng.random()
            if r < 0.4:
                self.lines.append(f"ldx{sz} r8 r0 {o}")
            elif r < 0.7:
                self.lines.append(f"stx{sz} r0 {o} r7")
            else:
                asz = [4, 8][self.i(0, 2)]
                self.lines += ["mov r3 1", f"atomic{asz} add r0 {self.off(vs, asz)} r3"]
            if skip:
                self.lines.append(f"{skip}:")
            self.lines.append(f"{out}:")
        elif k == 4:  # ring reservation
            size = [8, 16, 24, 40][self.i(0, 4)]
            out = self.lab()
            self.lines += ["ld_map r1 2", f"mov r2 {size}", "mov r3 0", "call ringbuf_reserve"]
            if self.rng.random() < 0.9:
                self.lines.append(f"jeq r0 0 {out}")
            self.lines.append(f"stx{sz} r0 {self.off(size, sz)} r7")
            r = self.rng.random()
            if r < 0.45:
                self.lines += ["mov r1 r0", "mov r2 0", "call ringbuf_submit"]
            elif r < 0.9:
                self.lines += ["mov r1 r0", "mov r2 0", "call ringbuf_discard"]
            self.lines.append(f"{out}:")
        elif k == 5:  # ring output of stack bytes, or of map-value bytes
            n = [8, 16, 24][self.i(0, 3)]
            if self.rng.random() < 0.5:
                self.lines += ["ld_map r1 2", "mov r2 r10", f"add r2 {-self.off(32, 8) - n}", f"mov r3 {n}",
                               "mov r4 0", "call ringbuf_output"]
            else:  # the helper reads n bytes of an array value from a (maybe variable) offset
                out = self.lab()
                self.lines += ["st4 r10 -4 1", "ld_map r1 0", "mov r2 r10", "add r2 -4", "call map_lookup_elem",
                               f"jeq r0 0 {out}", "mov r2 r0"]
                skip = self.variable_offset("r2", 24) if self.rng.random() < 0.5 else None
                if not skip:
                    self.lines.append(f"add r2 {self.off(24, 8)}")
                self.lines += ["ld_map r1 2", f"mov r3 {n}", "mov r4 0", "call ringbuf_output"]
                if skip:
                    self.lines.append(f"{skip}:")
                self.lines.append(f"{out}:")
        elif k == 6:  # a bounded or unbounded loop, or one whose state comes back unchanged
            lp = self.lab()
            if self.rng.random() < 0.15:
                self.lines += [f"{lp}:", "ldx8 r5 r6 16", f"jgt r5 {self.i(0, 300)} {lp}"]
            else:
                bound = self.i(1, 9) if self.rng.random() < 0.9 else "r7"
                self.lines += ["mov r5 0", f"{lp}:", "add r5 1", f"jlt r5 {bound} {lp}"]
        elif k == 7:  # variable stack offset
            self.lines += ["mov r2 r10", "add r2 -32"]
            skip = self.variable_offset("r2", 24)
            self.lines.append(f"stx{sz} r2 0 r7")
            if skip:
                self.lines.append(f"{skip}:")
        else:
            self.lines.append(f"{['add', 'xor', 'mul', 'rsh'][self.i(0, 4)]} r{self.i(7, 9)} {self.i(0, 9)}")

    def program(self):
        for _ in range(self.i(2, 7)):
            self.block()
        self.lines += ["mov r0 0", "exit"]
        return self.lines


def test_accepted_programs_never_fault():
    rng = np.random.default_rng(4242)
    accepted = 0
    for i in range(3000):
        lines = Gen(rng).program()
        try:
            prog = assemble(lines).prog()
        except Exception:  # an encoding the assembler refuses (e.g. an offset out of range)
            continue
        if gx.verify(prog, SPECS, CTX)[0] != 0:
            continue
        accepted += 1
        ev = rng.integers(0, 2**64 - 1, size=(64, CTX // 8), dtype=np.uint64, endpoint=True)
        ev[::3] &= np.uint64(0xFF)  # small values take the checked branches too
        try:  # the step budget is 2^20 per event: accepted loops are bounded far below it
            O.run(prog, O.maps_from_specs(SPECS), ev, CTX, strict_align=True)
        except O.OracleError as e:
            raise AssertionError((i, e, lines))
    assert accepted >= 300, accepted
