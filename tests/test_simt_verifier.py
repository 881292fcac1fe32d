"""SIMT-aware verification (gx_verify_simt): the warp-uniformity rules and per-hook budgets
of Sec. 4.4.1 and Sec. 5.3, host only.

The oracle's warp run (tests/test_oracle_warps.py) is the reference:
- every program it shows diverging is rejected at the instruction where its lanes disagree,
  with the matching reason;
- random warp handlers the pass accepts never diverge there (soundness);
- the budget counts bound the instructions the oracle executes per warp.
"""
import numpy as np
import pytest

import oracle as O
from tests.asmtext import assemble
from tests.test_oracle_warps import ARR, DIVERGING, HASH, RING, UNI, lookup0, warp_events
from workloads import gen
from workloads import programs as P

gx = pytest.importorskip("paper_2512_12615_gb300")

REASON = {"branch": gx.SIMT_V_BRANCH, "key": gx.SIMT_V_KEY, "atomic": gx.SIMT_V_ATOMIC, "store": gx.SIMT_V_STORE,
          "payload": gx.SIMT_V_HELPER, "exit": gx.SIMT_V_RET, "atomic_max": gx.SIMT_V_ATOMIC}


def simt(lines, specs, uniform, ctx_size=16, **kw):
    return gx.verify_simt(assemble(lines).prog(), specs, ctx_size, uniform, **kw)


@pytest.mark.parametrize("case", sorted(DIVERGING))
def test_rejected_where_the_oracle_diverges(case):
    lines, specs, pc = DIVERGING[case]
    rc, rep, log = simt(lines, specs, UNI)
    assert rc == gx.E_VERIFY and rep.violation == REASON[case] and rep.violation_pc == pc, log
    # the same program is fine when every ctx byte is warp-uniform, and when it runs per lane
    rc, rep, log = simt(lines, specs, np.ones(16, bool))
    assert rc == 0 and rep.violation == gx.SIMT_V_NONE and rep.violation_pc == -1, log
    assert gx.verify(assemble(lines).prog(), specs, 16)[0] == 0


def accepted(lines, specs, uniform=UNI, ctx_size=16):
    rc, rep, log = simt(lines, specs, uniform, ctx_size)
    assert rc == 0, log
    return rep


def rejected(lines, specs, why, pc, uniform=UNI, ctx_size=16):
    rc, rep, log = simt(lines, specs, uniform, ctx_size)
    assert rc == gx.E_VERIFY and (rep.violation, rep.violation_pc) == (why, pc), (rep.violation, rep.violation_pc, log)
    return log


def test_aggregated_values_are_uniform():
    """The program of the oracle's aggregation pin: a warp count of lane-varying bits added at
    a uniform key.  The oracle runs it without divergence."""
    lines = ["mov r9 r1", "ldx8 r1 r9 8", "and r1 1", "call warp_count", "mov r6 r0", "ldx8 r7 r9 0"] + lookup0() + [
        "jeq r0 0 out", "atomic8 add r0 0 r6", "out:", "mov r0 0", "exit"]
    rep = accepted(lines, ARR)
    assert rep.uniform_branches == 1 and rep.varying_insns == 2  # the lane address and its low bit
    O.run_warps(assemble(lines).prog(), O.maps_from_specs(ARR), warp_events(32, 4, seed=1), 16, uniform=UNI)


@pytest.mark.parametrize("helper", ["warp_sum_u64", "warp_max_u64", "warp_min_u64", "warp_or_u64", "warp_and_u64",
                                    "warp_count"])
def test_every_warp_helper_yields_a_uniform_key(helper):
    lines = ["ldx8 r1 r1 8", f"call {helper}", "stx8 r10 -8 r0", "stx8 r10 -16 r0", "ld_map r1 0", "mov r2 r10",
             "add r2 -8", "mov r3 r10", "add r3 -16", "mov r4 0", "call map_update_elem", "mov r0 0", "exit"]
    accepted(lines, HASH)
    # without the reduction the key is lane-varying
    rejected([lines[0], "mov r0 r1"] + lines[2:], HASH, gx.SIMT_V_KEY, 11)


def test_warp_helpers_are_refused_per_lane():
    rc, log = gx.verify(assemble(["mov r1 1", "call warp_sum_u64", "exit"]).prog(), [], 16)
    assert rc == gx.E_VERIFY and "unknown helper" in log


def test_lookup_and_delete_keys():
    rejected(["ldx8 r7 r1 8"] + lookup0() + ["mov r0 0", "exit"], ARR, gx.SIMT_V_KEY, 6)
    accepted(["ldx8 r7 r1 0"] + lookup0() + ["mov r0 0", "exit"], ARR)
    dele = ["ldx8 r7 r1 8", "stx8 r10 -8 r7", "ld_map r1 0", "mov r2 r10", "add r2 -8", "call map_delete_elem",
            "mov r0 0", "exit"]
    rejected(dele, HASH, gx.SIMT_V_KEY, 6)


def test_update_value_and_flags():
    upd = ["ldx8 r6 r1 0", "ldx8 r7 r1 8", "stx8 r10 -8 r6", "stx8 r10 -16 r7", "ld_map r1 0", "mov r2 r10",
           "add r2 -8", "mov r3 r10", "add r3 -16", "mov r4 0", "call map_update_elem", "mov r0 0", "exit"]
    rejected(upd, HASH, gx.SIMT_V_HELPER, 11)  # uniform key, lane-varying value
    flags = ["ldx8 r6 r1 0", "ldx8 r7 r1 8", "and r7 1", "stx8 r10 -8 r6", "stx8 r10 -16 r6", "ld_map r1 0",
             "mov r2 r10", "add r2 -8", "mov r3 r10", "add r3 -16", "mov r4 r7", "call map_update_elem", "mov r0 0",
             "exit"]
    rejected(flags, HASH, gx.SIMT_V_HELPER, 12)


def test_lane_varying_address_into_a_map_value():
    lines = (["ldx8 r6 r1 8", "and r6 8", "ldx8 r7 r1 0"] + lookup0() +
             ["jeq r0 0 out", "add r0 r6", "stx8 r0 0 r7", "out:", "mov r0 0", "exit"])
    rejected(lines, [dict(type=2, key_size=4, value_size=16, max_entries=4)], gx.SIMT_V_STORE, 11)
    atom = lines[:-4] + ["mov r2 1", "atomic8 add r0 0 r2", "out:", "mov r0 0", "exit"]
    rejected(atom, [dict(type=2, key_size=4, value_size=16, max_entries=4)], gx.SIMT_V_ATOMIC, 12)


def test_loop_bound():
    bounded = ["ldx8 r2 r1 8", "and r2 7", "mov r3 0", "mov r0 0", "l:", "add r0 1", "add r3 1", "jlt r3 r2 l", "exit"]
    rejected(bounded, [], gx.SIMT_V_BRANCH, 6)
    accepted(["ldx8 r2 r1 0", "and r2 7", "mov r3 0", "mov r0 0", "l:", "add r0 1", "add r3 1", "jlt r3 r2 l",
              "exit"], [])


def test_constants_are_uniform():
    """A value the verifier pins to one constant is the same in every lane."""
    accepted(["ldx8 r2 r1 8", "and r2 0", "mov r0 0", "jeq r2 0 out", "mov r0 1", "out:", "exit"], [])
    accepted(["ldx8 r2 r1 8", "mul r2 0", "mov r0 r2", "exit"], [])
    rejected(["ldx8 r2 r1 8", "and r2 1", "mov r0 r2", "exit"], [], gx.SIMT_V_RET, 3)


def test_marks_follow_the_stack():
    # a spilled lane-varying value stays lane-varying, whole or in part
    rejected(["ldx8 r2 r1 8", "stx8 r10 -8 r2", "ldx8 r0 r10 -8", "exit"], [], gx.SIMT_V_RET, 3)
    rejected(["ldx8 r2 r1 8", "stx8 r10 -8 r2", "ldx1 r0 r10 -6", "exit"], [], gx.SIMT_V_RET, 3)
    rejected(["ldx4 r2 r1 8", "stx4 r10 -8 r2", "ldx4 r0 r10 -8", "exit"], [], gx.SIMT_V_RET, 3)
    # uniform bytes written over varying ones are uniform again
    accepted(["ldx8 r2 r1 8", "stx8 r10 -8 r2", "ldx8 r3 r1 0", "stx8 r10 -8 r3", "ldx8 r0 r10 -8", "exit"], [])
    # an atomic on the lane's own stack is lane-private: allowed, and its result varies
    rejected(["st8 r10 -8 0", "ldx8 r2 r1 8", "atomic8 add r10 -8 r2", "ldx8 r0 r10 -8", "exit"], [],
             gx.SIMT_V_RET, 4)
    accepted(["st8 r10 -8 0", "ldx8 r2 r1 0", "atomic8 add r10 -8 r2", "ldx8 r0 r10 -8", "exit"], [])


def test_uniform_results_of_shared_state():
    """Helper results, values loaded through a uniform pointer and fetched old values are
    uniform (one execution per warp, broadcast)."""
    lines = (["ldx8 r7 r1 0"] + lookup0() +
             ["jeq r0 0 out", "mov r2 1", "atomic8 add_fetch r0 0 r2", "ldx8 r3 r0 0", "mov r0 0", "jgt r2 r3 out",
              "mov r0 r3", "out:", "exit"])
    rep = accepted(lines, ARR)
    assert rep.uniform_branches == 2 and rep.varying_insns == 0


def test_ring_buffer_records():
    res = ["ldx8 r6 r1 8", "ld_map r1 0", "mov r2 8", "mov r3 0", "call ringbuf_reserve", "jeq r0 0 out",
           "stx8 r0 0 r6", "mov r1 r0", "mov r2 0", "call ringbuf_submit", "out:", "mov r0 0", "exit"]
    rejected(res, RING, gx.SIMT_V_STORE, 7)
    accepted(["ldx8 r6 r1 0"] + res[1:], RING)


def test_uniform_flags_cover_the_ctx():
    with pytest.raises(ValueError):
        simt(["mov r0 0", "exit"], [], [True] * 15)


# ---------------------------------------------------------------- budgets (Sec. 5.3)
def budget(lines, specs=(), uniform=UNI, **kw):
    rc, rep, log = simt(lines, list(specs), uniform, **kw)
    return rc, rep, log


def test_budget_counts_are_path_maxima():
    rc, rep, _ = budget(["mov r0 0", "exit"])
    assert rc == 0 and (rep.max_insns, rep.max_helper_calls, rep.max_mem_ops) == (2, 0, 0)
    rc, rep, _ = budget(["ld_imm64 r0 5", "exit"])
    assert rc == 0 and rep.max_insns == 2  # a 64-bit immediate is one instruction
    # a diamond: 4 instructions one way, 7 the other
    diamond = ["ldx8 r2 r1 0", "jeq r2 0 l", "mov r0 1", "mov r0 2", "mov r0 3", "l:", "mov r0 0", "exit"]
    rc, rep, _ = budget(diamond)
    assert rc == 0 and (rep.max_insns, rep.max_mem_ops, rep.uniform_branches) == (7, 1, 1)
    # a loop of 8 trips: 1 + 8 * 2 + 2
    loop = ["mov r2 0", "l:", "add r2 1", "jlt r2 8 l", "mov r0 0", "exit"]
    rc, rep, _ = budget(loop)
    assert rc == 0 and rep.max_insns == 19
    rc, rep, log = budget(loop, max_insns=18)
    assert rc == gx.E_VERIFY and rep.violation == gx.SIMT_V_INSNS and rep.violation_pc == 4, log
    assert budget(loop, max_insns=19)[0] == 0


def test_helper_and_memory_budgets():
    lines = (["ldx8 r7 r1 0", "ldx8 r6 r1 0"] + lookup0() +
             ["jeq r0 0 out", "mov r1 r0", "mov r2 r6", "call atomic_max_u64", "out:", "mov r0 0", "exit"])
    rc, rep, _ = budget(lines, ARR)
    assert rc == 0 and (rep.max_helper_calls, rep.max_mem_ops) == (2, 3)
    rc, rep, log = budget(lines, ARR, max_helper_calls=1)
    assert rc == gx.E_VERIFY and (rep.violation, rep.violation_pc) == (gx.SIMT_V_HELPERS, 11), log
    rc, rep, log = budget(lines, ARR, max_mem_ops=2)
    assert rc == gx.E_VERIFY and (rep.violation, rep.violation_pc) == (gx.SIMT_V_MEM, 2), log
    assert budget(lines, ARR, max_helper_calls=2, max_mem_ops=3)[0] == 0


def test_ordinary_failures_are_reported():
    rc, rep, log = budget(["ldx8 r0 r10 -8", "exit"])
    assert rc == gx.E_VERIFY and rep.violation == gx.SIMT_V_VERIFY and rep.violation_pc == 0
    assert "uninitialised" in log


def per_warp_max_insns(prog, specs, ev, cs, uniform, lanes=32):
    most = 0
    maps = O.maps_from_specs(specs)
    for w0 in range(0, len(ev), lanes):
        _, c = O.run_warps(prog, maps, ev[w0:w0 + lanes], cs, uniform=uniform, lanes=lanes)
        most = max(most, c)
    return most


@pytest.mark.parametrize("name", ["counting", "page_heat", "latency"] + [f"random{p}" for p in range(0, 64, 3)])
def test_every_workload_program_is_a_uniform_handler(name):
    """With every ctx byte uniform nothing is lane-varying: each program the engine runs is
    accepted, and its instruction maximum bounds what the oracle executes per event."""
    if name == "counting":
        (prog, specs, cs), ev = P.counting(), gen.uniform_events(500, seed=1)
    elif name == "page_heat":
        (prog, specs, cs), ev = P.page_heat(), gen.pageheat_events(500, seed=2)
    elif name == "latency":
        (prog, specs, cs), ev = P.latency(ring_bytes=1 << 16), gen.latency_pairs(500, seed=3)
    else:
        p = int(name[6:])
        (prog, specs, cs), ev = P.batch_programs()[p], gen.uniform_events(300, seed=10 + p)
    rc, rep, log = gx.verify_simt(prog, specs, cs, np.ones(cs, bool))
    assert rc == 0 and rep.varying_insns == 0, log
    raw = np.ascontiguousarray(ev).view(np.uint8).reshape(-1, cs)
    assert 0 < per_warp_max_insns(prog, specs, raw, cs, None, lanes=1) <= rep.max_insns


# ---------------------------------------------------------------- soundness against the oracle
def random_handler(rng):
    """A random warp handler over a 32-byte ctx: loads, ALU work, warp reductions, uniform or
    lane-varying branches, map updates, map-value atomics, ring-buffer output and R0.  Safe
    for the ordinary verifier; whether it is warp-uniform depends on the ctx mask."""
    regs = ["r6", "r7", "r8"]
    lines = ["mov r9 r1"] + [f"ldx8 {r} r9 {8 * int(rng.integers(0, 4))}" for r in regs]
    label = 0
    for _ in range(int(rng.integers(3, 9))):
        a, b = (regs[int(i)] for i in rng.integers(0, 3, 2))
        k = int(rng.integers(0, 9))
        if k == 0:
            lines.append(f"ldx8 {a} r9 {8 * int(rng.integers(0, 4))}")
        elif k == 1:
            op = ["add", "xor", "or", "and", "mul", "sub"][int(rng.integers(0, 6))]
            lines.append(f"{op} {a} {b}")
        elif k == 2:
            lines.append(["and {} 15", "rsh {} 3", "add {} 7", "and {} 0"][int(rng.integers(0, 4))].format(a))
        elif k == 3:
            h = ["warp_sum_u64", "warp_max_u64", "warp_min_u64", "warp_or_u64", "warp_and_u64", "warp_count"]
            lines += [f"mov r1 {a}", f"call {h[int(rng.integers(0, 6))]}", f"mov {b} r0"]
        elif k == 4:
            label += 1
            lines += [f"jgt {a} {int(rng.integers(0, 16))} s{label}", f"add {b} 1", f"s{label}:"]
        elif k == 5:
            lines += [f"stx8 r10 -8 {a}", f"stx8 r10 -16 {b}", "ld_map r1 0", "mov r2 r10", "add r2 -8",
                      "mov r3 r10", "add r3 -16", "mov r4 0", "call map_update_elem"]
        elif k == 6:
            label += 1
            lines += [f"mov r5 {a}", "and r5 7", "stx4 r10 -4 r5", "ld_map r1 1", "mov r2 r10", "add r2 -4",
                      "call map_lookup_elem", f"jeq r0 0 s{label}", f"atomic8 add r0 0 {b}", f"s{label}:"]
        elif k == 7:
            lines += [f"stx8 r10 -24 {a}", "ld_map r1 2", "mov r2 r10", "add r2 -24", "mov r3 8", "mov r4 0",
                      "call ringbuf_output"]
        else:
            label += 1
            lines += ["mov r5 0", f"l{label}:", f"add {a} 1", "add r5 1", f"jlt r5 3 l{label}"]
    lines += [f"mov r0 {regs[int(rng.integers(0, 3))]}" if rng.random() < 0.5 else "mov r0 0", "exit"]
    return lines


RANDOM_SPECS = [dict(type=1, key_size=8, value_size=8, max_entries=4096), dict(type=2, key_size=4, value_size=8,
                max_entries=8), dict(type=27, key_size=0, value_size=0, max_entries=1 << 16)]


def random_warps(rng, uniform_words, warps=4, lanes=32, tail=11):
    n = warps * lanes + tail
    ev = np.zeros((n, 4), dtype=np.uint64)
    small = rng.random(4) < 0.5  # small values make branches, keys and slots collide
    for w in range(4):
        hi = 16 if small[w] else 1 << 40
        lane_vals = rng.integers(0, hi, size=n, dtype=np.uint64)
        if uniform_words[w]:
            warp_vals = rng.integers(0, hi, size=warps + 1, dtype=np.uint64)
            lane_vals = np.repeat(warp_vals, lanes)[:n]
        ev[:, w] = lane_vals
    return ev


def test_accepted_handlers_never_diverge():
    """Soundness: over 400 random handlers and ctx masks, every program the pass accepts runs
    through the oracle's warp run without a disagreement, with per-warp instruction counts
    within the reported maximum; and the rejected ones mostly do diverge there."""
    rng = np.random.default_rng(2024)
    n_acc = n_rej = n_witness = 0
    for i in range(400):
        lines = random_handler(rng)
        words = rng.random(4) < 0.5
        uniform = np.repeat(words, 8)
        prog = assemble(lines).prog()
        rc, rep, log = gx.verify_simt(prog, RANDOM_SPECS, 32, uniform)
        assert rc == 0 or rep.violation not in (gx.SIMT_V_NONE, gx.SIMT_V_VERIFY), (i, log, lines)
        ev = random_warps(rng, words)
        if rc == 0:
            n_acc += 1
            most = per_warp_max_insns(prog, RANDOM_SPECS, ev, 32, uniform)
            assert most <= rep.max_insns, (i, lines)
        else:
            n_rej += 1
            try:
                O.run_warps(prog, O.maps_from_specs(RANDOM_SPECS), ev, 32, uniform=uniform)
            except O.OracleError as e:
                assert e.rc == O.EDIVERGE, (i, e, lines)
                n_witness += 1
    assert n_acc >= 80 and n_rej >= 80, (n_acc, n_rej)
    assert n_witness >= 0.6 * n_rej, (n_witness, n_rej)


def test_warp_heat_budgets_and_their_worst_path():
    """The warp-level policy is a uniform handler over warp-context records.  Its worst path
    (a valid warp that inserts its region and has misaligned lanes) runs 82 instructions,
    12 helper calls and 19 memory operations, counted by hand along the program; the oracle
    reaches exactly 82 on such a warp."""
    prog, specs, cs = P.warp_heat()
    rc, rep, log = gx.verify_simt(prog, specs, cs, gen.WARP_UNIFORM)
    assert rc == 0, log
    assert (rep.max_insns, rep.max_helper_calls, rep.max_mem_ops) == (82, 12, 19)
    assert gx.verify_simt(prog, specs, cs, gen.WARP_UNIFORM, max_insns=81)[1].violation == gx.SIMT_V_INSNS
    assert gx.verify_simt(prog, specs, cs, gen.WARP_UNIFORM, max_insns=82, max_helper_calls=12, max_mem_ops=19)[0] == 0
    # the per-lane engine refuses its warp helpers; with the address also declared uniform
    # nothing varies
    assert gx.verify(prog, specs, cs)[0] == gx.E_VERIFY
    assert gx.verify_simt(prog, specs, cs, np.ones(cs, bool))[1].varying_insns == 0
    ev = gen.warp_access_events(200, seed=4)
    ev["addr"][::3] |= np.uint64(1)  # misaligned lanes in every warp
    raw = np.ascontiguousarray(ev).view(np.uint8).reshape(-1, cs)
    assert per_warp_max_insns(prog, specs, raw, cs, gen.WARP_UNIFORM) == 82
    # with the address lane-varying and no reduction in between, its region would be a key
    lines = ["ldx8 r7 r1 0", "rsh r7 21", "stx8 r10 -8 r7", "ld_map r1 0", "mov r2 r10", "add r2 -8",
             "call map_lookup_elem", "mov r0 0", "exit"]
    rejected(lines, specs, gx.SIMT_V_KEY, 7, uniform=gen.WARP_UNIFORM, ctx_size=32)


def test_all_uniform_simt_mode_judges_like_the_per_lane_verifier():
    """With every ctx byte uniform nothing is lane-varying, so SIMT mode (path counters and
    the pruning they restrict included) must accept and reject exactly what the per-lane
    verifier does, for the same reason, over the memory-safety fuzzer's random programs; and
    the instruction, helper-call and memory-operation maxima it reports bound what any event
    of an accepted program executes on the oracle."""
    from tests.test_verifier_fuzz import CTX, SPECS as FSPECS, Gen

    rng = np.random.default_rng(777)
    both = 0
    for _ in range(500):
        prog = assemble(Gen(rng).program()).prog()
        rc1, log1 = gx.verify(prog, FSPECS, CTX)
        rc2, rep, log2 = gx.verify_simt(prog, FSPECS, CTX, np.ones(CTX, bool))
        # the same verdict for the same reason; exploring in another order may stop elsewhere
        assert rc1 == rc2 and log1.split(": ", 1)[-1] == log2.split(": ", 1)[-1], (log1, log2)
        if rc1 == 0:
            both += 1
            assert rep.varying_insns == 0 and rep.max_insns > 0
            # the reported path maxima bound what any event executes
            ev = rng.integers(0, 2**64 - 1, size=(32, CTX // 8), dtype=np.uint64, endpoint=True)
            ev[::3] &= np.uint64(0xFF)
            most = []
            O.run(prog, O.maps_from_specs(FSPECS), ev, CTX, most=most)
            assert most[0] <= rep.max_insns and most[1] <= rep.max_helper_calls and most[2] <= rep.max_mem_ops, \
                (most, rep.max_insns, rep.max_helper_calls, rep.max_mem_ops)
        else:
            assert rep.violation == gx.SIMT_V_VERIFY
    assert both >= 60
