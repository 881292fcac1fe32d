"""The verifier's "combinable" classification (gx_analyze), fuzzed on the oracle.

Block-private combining (the hierarchical maps of Sec. 5.3) holds a combinable map's
updates back in shared memory and merges them later, so it is invisible only if the program
never looks at those values.  The oracle's deferral mode takes that to the extreme: the
updates of the deferred maps are applied after the last event, and any other use of their
values stops the run (EDEFER).  For every map gx_analyze calls combinable in a random
program, the deferred run must equal the plain one: maps, ring payloads, every R0.
"""
import numpy as np
import pytest

import oracle as O
from tests.asmtext import assemble
from tests.test_det_fuzz import SPECS, Gen

gx = pytest.importorskip("paper_2512_12615_gb300")


class CGen(Gen):
    """The determinism fuzzer's programs, plus uses of map values through helpers: ring
    output straight from a value, a lookup keyed by value bytes, an overwriting update."""

    def block(self, depth=0):
        r = self.rng.random()
        if r >= 0.2:
            return super().block(depth)
        skip = self.fresh()
        self.array_value(skip)
        if r < 0.07:
            self.lines += ["mov r2 r0", "ld_map r1 2", "mov r3 8", "mov r4 0", "call ringbuf_output"]
        elif r < 0.14:
            self.lines += ["mov r2 r0", "ld_map r1 1", "call map_lookup_elem"]
        else:
            self.lines += [f"stx8 r10 -8 {self.r()}", "st8 r10 -24 0", "st8 r10 -16 0", "ld_map r1 0",
                           "mov r2 r10", "add r2 -4", "mov r3 r10", "add r3 -24", "mov r4 0",
                           "call map_update_elem"]
        self.lines.append(f"{skip}:")


def outcome(prog, ev, defer):
    maps = O.maps_from_specs(SPECS)
    r0, _ = O.run(prog, maps, ev, 32, want_r0=True, defer_maps=defer)
    recs, dropped = maps[2].ringbuf_records()
    return maps[0].array_values().tobytes(), sorted(maps[1].hash_items().items()), recs, dropped, r0.tolist()


def test_combinable_maps_can_be_deferred():
    rng = np.random.default_rng(5150)
    deferred = 0
    for i in range(2000):
        lines = CGen(rng).program()
        prog = assemble(lines).prog()
        rc, info, _ = gx.analyze(prog, SPECS, 32)
        if rc != 0 or not info.combinable_maps:
            continue
        deferred += 1
        ev = rng.integers(0, 12, size=(200, 4), dtype=np.uint64)
        ev[::5] = rng.integers(0, 2**40, size=(len(ev[::5]), 4), dtype=np.uint64)
        plain = outcome(prog, ev, 0)
        try:
            late = outcome(prog, ev, info.combinable_maps)
        except O.OracleError as e:
            raise AssertionError((i, "a map called combinable is used otherwise", e, lines))
        assert late == plain, (i, lines)
    assert deferred >= 300, deferred


def test_deferral_catches_an_observed_map():
    """A program that reads back the value it adds to: deferring that map is refused."""
    lines = ["st4 r10 -4 0", "ld_map r1 0", "mov r2 r10", "add r2 -4", "call map_lookup_elem", "jeq r0 0 out",
             "mov r1 1", "atomic8 add r0 0 r1", "ldx8 r1 r0 0", "out:", "mov r0 0", "exit"]
    prog = assemble(lines).prog()
    rc, info, _ = gx.analyze(prog, SPECS, 32)
    assert rc == 0 and info.combinable_maps == 0
    with pytest.raises(O.OracleError) as e:
        O.run(prog, O.maps_from_specs(SPECS), np.zeros((3, 4), np.uint64), 32, defer_maps=1)
    assert e.value.rc == O.EDEFER
    # without the read-back the map is combinable and deferring it changes nothing
    prog = assemble(lines[:8] + lines[9:]).prog()
    rc, info, _ = gx.analyze(prog, SPECS, 32)
    assert rc == 0 and info.combinable_maps == 1
    assert outcome(prog, np.zeros((3, 4), np.uint64), 1) == outcome(prog, np.zeros((3, 4), np.uint64), 0)
