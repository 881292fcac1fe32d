"""Host-only: every workload program specialises and compiles for sm_103a (no device needed)."""
import pytest

import paper_2512_12615_gb300 as gx
from tests.asmtext import assemble
from workloads import programs as P


def _check(prog, specs, cs, det=True):
    rc, log = gx.jit_check(prog, specs, cs, deterministic=det)
    if rc == gx.E_NODEV:
        pytest.skip("no runtime compiler on this host")
    assert rc == 0, log


@pytest.mark.parametrize("build", [P.counting, P.page_heat, P.latency])
def test_workload_programs_compile(build):
    _check(*build())


@pytest.mark.parametrize("p", [0, 21, 63])
def test_batch_programs_compile(p):
    _check(*P.batch_programs()[p])


def test_rejected_program_is_not_compiled():
    rc, log = gx.jit_check(assemble(["ldx8 r0 r10 -8", "exit"]).prog(), [], 16)
    assert rc == gx.E_VERIFY and "uninitialised stack" in log


# ---------------------------------------------------------------- combining layouts (compile only)
def _hash_upd(m, ks, vs, key_expr, body):
    """lookup-or-insert in hash map m (key in r7 after key_expr), then body on r0 (non-NULL)"""
    ins = [f"mov r7 {key_expr[0]}", f"and r7 {key_expr[1]}", f"stx{ks} r10 -8 r7", f"ld_map r1 {m}", "mov r2 r10",
           "add r2 -8", "call map_lookup_elem", f"jne r0 0 have{m}"]
    ins += [f"st8 r10 {-8 - 8 * (k + 1)} 0" for k in range(vs // 8)]
    ins += [f"ld_map r1 {m}", "mov r2 r10", "add r2 -8", "mov r3 r10", f"add r3 {-8 - vs}", "mov r4 1",
            "call map_update_elem", f"ld_map r1 {m}", "mov r2 r10", "add r2 -8", "call map_lookup_elem",
            f"jeq r0 0 out{m}", f"have{m}:"] + body + [f"out{m}:"]
    return ins


def _arr_upd(m, n, body):
    return ["mov r7 r8", f"and r7 {n - 1}", "stx4 r10 -4 r7", f"ld_map r1 {m}", "mov r2 r10", "add r2 -4",
            "call map_lookup_elem", f"jeq r0 0 aout{m}"] + body + [f"aout{m}:"]


MANY = (["mov r6 r1", "ldx8 r8 r6 8"]
        + _hash_upd(0, 8, 24, ("r8", "0xFF"), ["mov r9 r0", "mov r1 r8", "atomic8 add r0 0 r1", "mov r1 r9",
                                                  "add r1 8", "mov r2 r8", "call atomic_max_u64", "mov r0 r9",
                                                  "mov r1 r8", "atomic4 xor r0 16 r1", "atomic4 or r0 20 r1"])
        + _hash_upd(1, 8, 248, ("r8", "0x3F"), ["mov r9 r0", "mov r1 r8", "atomic8 add r0 0 r1", "mov r1 r9",
                                                   "add r1 240", "mov r2 r8", "call atomic_min_u64"])
        + _arr_upd(2, 16, ["mov r1 r8", "atomic8 and r0 0 r1"])
        + _arr_upd(3, 1024, ["mov r1 r8", "atomic8 or r0 0 r1", "atomic4 add r0 8 r1"])
        + ["mov r0 0", "exit"])
MANY_SPECS = [dict(type=1, key_size=8, value_size=24, max_entries=512, flags=1),
              dict(type=1, key_size=8, value_size=248, max_entries=128),
              dict(type=2, key_size=4, value_size=8, max_entries=16),
              dict(type=2, key_size=4, value_size=16, max_entries=1024)]  # 16 KiB: above the copy limit, cached


def test_many_maps_compile_and_combine():
    prog = assemble(MANY).prog()
    rc, info, log = gx.analyze(prog, MANY_SPECS, 32, deterministic=True)
    assert rc == 0, log
    assert info.combinable_maps == 0b1111
    _check(prog, MANY_SPECS, 32)


def test_stack_at_varying_offsets_compiles():
    # one store reaches two stack slots on different paths: the stack stays in memory
    lines = ["ldx8 r2 r1 0", "mov r3 r10", "add r3 -8", "jeq r2 0 a", "mov r3 r10", "add r3 -16", "a:",
             "st8 r3 0 7", "st8 r10 -8 1", "st8 r10 -16 2", "ldx8 r0 r10 -8", "exit"]
    prog = assemble(lines).prog()
    assert gx.verify(prog, [], 16)[0] == 0
    _check(prog, [], 16, det=False)


def test_ring_output_from_scalar_stack_compiles():
    lines = ["ldx8 r2 r1 0", "stx8 r10 -16 r2", "st8 r10 -8 5", "ld_map r1 0", "mov r2 r10", "add r2 -16",
             "mov r3 16", "mov r4 0", "call ringbuf_output", "mov r0 0", "exit"]
    _check(assemble(lines).prog(), [dict(type=27, key_size=0, value_size=0, max_entries=4096)], 16, det=False)


# ---------------------------------------------------------------- warp-level form (compile only)
# ctx 32 bytes: word 0 lane-varying, words 1..3 warp-uniform
WARP_UNI = [False] * 8 + [True] * 24
EVERY_EFFECT = """
mov r9 r1
ldx8 r6 r9 0
ldx8 r7 r9 8
mov r1 r6
call warp_sum_u64
mov r8 r0
mov r1 r6
call warp_or_u64
add r8 r0
mov r1 r6
call warp_and_u64
add r8 r0
mov r1 r6
call warp_max_u64
add r8 r0
mov r1 r6
call warp_min_u64
add r8 r0
mov r1 r6
call warp_count
add r8 r0
st8 r10 -8 0
atomic8 add r10 -8 r6
mov r2 r10
add r2 -16
jeq r7 0 slot
mov r2 r10
add r2 -24
slot:
st8 r2 0 5
mov r1 r7
and r1 3
stx4 r10 -28 r1
ld_map r1 0
mov r2 r10
add r2 -28
call map_lookup_elem
jeq r0 0 skip
mov r5 r0
mov r1 r8
atomic8 add_fetch r5 0 r1
mov r1 7
atomic8 xchg r5 8 r1
mov r0 0
mov r1 9
atomic8 cmpxchg r5 16 r1
stx8 r5 24 r8
mov r1 r5
mov r2 r8
call atomic_min_u64
skip:
stx8 r10 -40 r7
stx8 r10 -48 r8
ld_map r1 1
mov r2 r10
add r2 -40
mov r3 r10
add r3 -48
mov r4 0
call map_update_elem
ld_map r1 1
mov r2 r10
add r2 -40
call map_delete_elem
ld_map r1 2
mov r2 16
mov r3 0
call ringbuf_reserve
jeq r0 0 one
stx8 r0 0 r8
st8 r0 8 1
mov r1 r0
mov r2 0
call ringbuf_submit
one:
ld_map r1 2
mov r2 8
mov r3 0
call ringbuf_reserve
jeq r0 0 two
mov r1 r0
mov r2 0
call ringbuf_discard
two:
stx8 r10 -56 r8
ld_map r1 2
mov r2 r10
add r2 -56
mov r3 8
mov r4 0
call ringbuf_output
mov r0 r8
exit
""".strip().splitlines()
EVERY_EFFECT_SPECS = [dict(type=2, key_size=4, value_size=32, max_entries=4),
                      dict(type=1, key_size=8, value_size=8, max_entries=64),
                      dict(type=27, key_size=0, value_size=0, max_entries=1 << 16)]


def _check_warp(prog, specs, cs, uniform):
    rc, log = gx.jit_check_simt(prog, specs, cs, uniform)
    if rc == gx.E_NODEV:
        pytest.skip("no runtime compiler on this host")
    assert rc == 0, log


def test_warp_form_of_every_shared_effect_compiles():
    """Helpers, fetches, exchanges, stores and ring-buffer records on the leader lane with
    their results broadcast; warp helpers; lane-private stack atomics; stack slots at
    path-dependent offsets (the addressable stack)."""
    import numpy as np

    import oracle as O
    from tests.test_simt_verifier import random_warps

    prog = assemble(EVERY_EFFECT).prog()
    rc, rep, log = gx.verify_simt(prog, EVERY_EFFECT_SPECS, 32, WARP_UNI)
    assert rc == 0 and rep.varying_insns > 0, log
    # the oracle's warp run takes it without a disagreement
    ev = random_warps(np.random.default_rng(3), [False, True, True, True])
    O.run_warps(prog, O.maps_from_specs(EVERY_EFFECT_SPECS), ev, 32, uniform=WARP_UNI)
    _check_warp(prog, EVERY_EFFECT_SPECS, 32, WARP_UNI)


def test_warp_form_of_warp_heat_compiles():
    from workloads import gen

    _check_warp(*P.warp_heat(), gen.WARP_UNIFORM)


def test_warp_form_of_random_handlers_compiles():
    import numpy as np

    from tests.test_simt_verifier import RANDOM_SPECS, random_handler

    rng = np.random.default_rng(77)
    done = 0
    while done < 3:
        lines = random_handler(rng)
        uniform = np.repeat(rng.random(4) < 0.5, 8)
        prog = assemble(lines).prog()
        if gx.verify_simt(prog, RANDOM_SPECS, 32, uniform)[0] != 0:
            continue
        _check_warp(prog, RANDOM_SPECS, 32, uniform)
        done += 1


def test_warp_form_needs_simt_verification():
    rc, log = gx.jit_check_simt(assemble(["ldx8 r0 r1 0", "exit"]).prog(), [], 16, [False] * 16)
    assert rc == gx.E_VERIFY and "lane-varying" in log


def _leader_regions(line: str):
    """The text inside each `if (lead) { ... }` and `if (!sh_ || lead) { ... }` of a line."""
    out = []
    for head in ("if (lead) {", "if (!sh_ || lead) {"):
        start = 0
        while (i := line.find(head, start)) >= 0:
            depth, j = 0, i + len(head) - 1
            while j < len(line):
                depth += {"{": 1, "}": -1}.get(line[j], 0)
                if depth == 0:
                    break
                j += 1
            out.append(line[i + len(head):j])
            start = j
    return out


def test_warp_form_keeps_collectives_out_of_leader_code(tmp_path, monkeypatch):
    """In the warp-level form only the leader runs helper calls and shared stores; a
    collective over the warp's lanes (wmask or the full mask) inside that code would wait
    for lanes that never come.  Collectives over __activemask() are fine there."""
    import re

    import numpy as np

    from tests.test_simt_verifier import RANDOM_SPECS, random_handler
    from workloads import gen

    monkeypatch.setenv("GX_JIT_DUMP_DIR", str(tmp_path))
    cases = [(assemble(EVERY_EFFECT).prog(), EVERY_EFFECT_SPECS, 32, WARP_UNI),
             (*P.warp_heat(), gen.WARP_UNIFORM)]
    rng = np.random.default_rng(5)
    while len(cases) < 6:
        uniform = np.repeat(rng.random(4) < 0.5, 8)
        prog = assemble(random_handler(rng)).prog()
        if gx.verify_simt(prog, RANDOM_SPECS, 32, uniform)[0] == 0:
            cases.append((prog, RANDOM_SPECS, 32, uniform))
    warp_wide = re.compile(r"(__shfl_sync|__ballot_sync|__syncwarp|__reduce_\w+_sync|group_reduce<[^>]*>)\(\s*"
                           r"(wmask|0x[fF]+u)")
    for prog, specs, cs, uniform in cases:
        _check_warp(prog, specs, cs, uniform)
    sources = list(tmp_path.glob("*.cu"))
    assert len(sources) >= len(cases) - 1  # identical programs share a source
    leader_lines = 0
    for f in sources:
        for line in f.read_text().splitlines():
            for region in _leader_regions(line):
                leader_lines += 1
                assert not warp_wide.search(region), (f.name, line)
    assert leader_lines > 20
    # every leader-only region is followed by a barrier of the warp's lanes before anything else
    for f in sources:
        for line in f.read_text().splitlines():
            for head in ("if (lead) {", "if (!sh_ || lead) {"):
                if head in line:
                    tail = line.split(head, 1)[1]
                    assert "__syncwarp(wmask);" in tail, (f.name, line)


def _structured_joins_are_safe(body: str, name: str) -> int:
    """In the structured (loop-free) form the only collectives are the ballot of the valid
    lanes, before any branch, and __syncwarp over those lanes between blocks, at the top
    level of the body; no valid lane returns before the end.  Returns the joins seen."""
    lines = body.splitlines()
    start = next(i for i, l in enumerate(lines) if l.startswith("__device__ __forceinline__ u64 gx_body_"))
    depth, joins, seen_valid_check, returns = 0, 0, False, []
    for line in lines[start:]:
        if "_sync(" in line or "__syncwarp" in line:
            if line.strip() == "const u32 vm_ = __ballot_sync(0xFFFFFFFFu, valid);":
                assert not seen_valid_check and depth == 1, (name, line)
            else:
                assert line.strip() == "__syncwarp(vm_);" and depth == 1, (name, line)
                joins += 1
        if line.strip() == "if (!valid) return 0;":
            seen_valid_check = True
        elif "return" in line:
            returns.append(line.strip())
        depth += line.count("{") - line.count("}")
        if depth == 0:
            break
    # the end of the body, and the budget trip that a loop-free program never reaches
    assert returns == ["return r0;", "return 0;"], (name, returns)
    return joins


def test_per_lane_form_has_no_collectives_of_its_own(tmp_path, monkeypatch):
    """Per-lane generated code runs after data-dependent branches, so a collective in it
    could wait for lanes on another path.  Programs with loops have none: warp cooperation
    happens inside the device helpers, under the mask of the lanes that called them
    (__activemask()).  Loop-free programs join their valid lanes between basic blocks, at
    points every valid lane passes (checked line by line)."""
    monkeypatch.setenv("GX_JIT_DUMP_DIR", str(tmp_path))
    progs = [P.counting(), P.page_heat(), P.latency()] + [P.batch_programs()[p] for p in (0, 9, 33, 63)]
    for prog, specs, cs in progs:
        _check(prog, specs, cs)
    _check(assemble(MANY).prog(), MANY_SPECS, 32)
    sources = list(tmp_path.glob("*.cu"))
    assert len(sources) == len(progs) + 1
    structured = 0
    for f in sources:
        body = f.read_text().split("} // namespace gx")[0]  # the program bodies, before the entry points
        if "u32 nb_ = 0;" in body:
            structured += 1
            assert _structured_joins_are_safe(body, f.name) > 0, f.name
        else:
            assert "_sync(" not in body and "__syncwarp" not in body, f.name
        assert "__activemask()" in body or "agg_update" not in body, f.name
    assert structured >= 5  # counting, latency, the generated programs; page-heat has a loop


# ---------------------------------------------------------------- work stealing (compile only)
SCHED_KINDS = ["fixed", "greedy", "latency_budget"]


def _check_sched(prog, specs, cs, hook, hook_specs, **kw):
    rc, log = gx.jit_check_sched(prog, specs, cs, hook, hook_specs, deterministic=True, **kw)
    if rc == gx.E_NODEV:
        pytest.skip("no runtime compiler on this host")
    assert rc == 0, log


@pytest.mark.parametrize("kind", SCHED_KINDS)
def test_stealing_kernel_compiles(kind):
    """The persistent kernel of mode 2 (shares, a scheduling program asked before each
    stolen chunk) compiles for sm_103a with each policy steering it."""
    hook, hook_specs, _ = P.sched_policy(kind)
    for build in (P.counting, P.page_heat):
        _check_sched(*build(), hook, hook_specs)
    _check_sched(*P.batch_programs()[9], hook, hook_specs)


def test_scheduling_program_must_qualify():
    """The hook context is 32 warp-uniform bytes; a program over the hook budget is refused
    with the budget named, and one with another context size is not a scheduling program."""
    prog, specs, cs = P.counting()
    hook, hook_specs, _ = P.sched_policy("latency_budget")  # worst path: 22 insns, 1 call, 7 memory ops
    rc, log = gx.jit_check_sched(prog, specs, cs, hook, hook_specs, max_insns=21)
    assert rc == gx.E_VERIFY, log
    rc, log = gx.jit_check_sched(prog, specs, cs, hook, hook_specs, max_mem_ops=6)
    assert rc == gx.E_VERIFY, log
    _check_sched(prog, specs, cs, hook, hook_specs, max_insns=22, max_helper_calls=1, max_mem_ops=7)
    # the scheduling program's context is GX_SCHED_CTX bytes: a 64-byte reader is not one
    reader = assemble(["ldx8 r0 r1 56", "exit"]).prog()
    rc, log = gx.jit_check_sched(prog, specs, cs, reader, [])
    assert rc == gx.E_VERIFY and "ctx" in log, log
    _check_sched(prog, specs, cs, assemble(["ldx8 r0 r1 24", "exit"]).prog(), [])  # the budget field


def test_stealing_source_shape(tmp_path, monkeypatch):
    """Only a batch with a scheduling program gets the stealing skeleton: its source holds
    one out-of-line scheduling call, the skeleton in every entry point, and the hook's body
    has no collective of its own.  Sources without one never include the header."""
    monkeypatch.setenv("GX_JIT_DUMP_DIR", str(tmp_path / "sched"))
    hook, hook_specs, _ = P.sched_policy("greedy")
    _check_sched(*P.page_heat(), hook, hook_specs)
    (src,) = list((tmp_path / "sched").glob("*.cu"))
    text = src.read_text()
    assert text.count('#include "gx_steal.cuh"') == 1
    assert text.count("__device__ __noinline__ u64 gx_sched_call(") == 1
    assert text.count("gx::exec_steal(P,") == 2 and "gx::exec_tiles(" not in text  # wide and capped entries
    assert text.count("__launch_bounds__(256, 2)") == 1 and text.count("__launch_bounds__(256, 5)") == 1
    body = "__device__ __forceinline__ u64 gx_body_1(" + text.split("__device__ __noinline__ u64 gx_sched_call(")[0].split(
        "gx_body_1(")[1]
    # the whole of warp 0 runs the hook (one lane valid); its only joins are the structured ones
    assert _structured_joins_are_safe(body, src.name) > 0
    monkeypatch.setenv("GX_JIT_DUMP_DIR", str(tmp_path / "plain"))
    _check(*P.page_heat())
    (plain,) = list((tmp_path / "plain").glob("*.cu"))
    ptext = plain.read_text()
    assert "gx_steal" not in ptext and "gx_sched_call" not in ptext and "exec_steal" not in ptext


def test_loop_free_joins_only_where_jumps_land(tmp_path, monkeypatch):
    """A block entered only by falling through has one way in, so it needs no warp join.
    The latency program's blocks are the fall-through side of its validation branches,
    except the shared exit block that every failed check jumps to: one join in all."""
    monkeypatch.setenv("GX_JIT_DUMP_DIR", str(tmp_path))
    prog, specs, cs = P.latency()
    _check(prog, specs, cs)
    (f,) = list(tmp_path.glob("*.cu"))
    body = f.read_text().split("} // namespace gx")[0]
    assert body.count("if (nb_ == ") == 10
    assert body.count("__syncwarp(vm_)") == 1
