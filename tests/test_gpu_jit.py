"""The load-time specialised (JIT) form against the oracle on the GPU: same bit-exact bar
as the interpreter, same programs, ragged sizes and launch shapes."""
import json
import os

import numpy as np
import pytest

from tests import closed_forms as CF
from tests.asmtext import assemble
from tests.parity import device_events, run_both
from workloads import gen
from workloads import programs as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    import paper_2512_12615_gb300 as gx

    return gx.Context(0)


@pytest.mark.parametrize("launch", [None, (64, 3), (256, 16)])
def test_counting_jit(ctx, launch):
    prog, specs, cs = P.counting()
    ev = gen.uniform_events(100_003, seed=31)
    gs, _, _, _ = run_both(ctx, prog, specs, cs, ev, jit=True, launch=launch)
    assert np.array_equal(gs[0][1].view("<u8")[:, 0], CF.counting(ev))


@pytest.mark.parametrize("n", [1, 33, 32 * 257 + 5, 200_001])
def test_page_heat_jit(ctx, n):
    prog, specs, cs = P.page_heat()
    ev = gen.pageheat_events(n, seed=32 + n)
    ev["size"][::97] = 3
    ev["kind"][5::101] = 9
    ev["addr"][7::89] |= np.uint64(1)
    run_both(ctx, prog, specs, cs, ev, jit=True)


def test_latency_jit(ctx):
    prog, specs, cs = P.latency(ring_bytes=1 << 22)
    ev = gen.latency_pairs(100_001, seed=33)
    gs, _, _, _ = run_both(ctx, prog, specs, cs, ev, jit=True)
    hist, outliers = CF.latency(ev)
    assert np.array_equal(gs[0][1].view("<u8")[:, 0], hist)
    assert gs[1][1] == outliers


@pytest.mark.parametrize("p", range(0, 64, 3))
def test_random_program_jit(ctx, p):
    prog, specs, cs = P.batch_programs()[p]
    run_both(ctx, prog, specs, cs, gen.uniform_events(20_000 + 37 * p, seed=300 + p), jit=True)


CASES = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "handworked.json")))["cases"]


@pytest.mark.parametrize("case", [c for c in CASES if c["name"] != "ringbuf_full_drops" and "oracle_only" not in c],
                         ids=lambda c: c["name"])
def test_handworked_jit(ctx, case):
    specs = [dict(m) for m in case.get("maps", [])]
    for m in specs:
        if m["type"] == 27:
            m["max_entries"] = max(4096, m["max_entries"])
    ev = np.array(case["events"], dtype=np.uint64)
    _, _, r0, _ = run_both(ctx, assemble(case["asm"]).prog(), specs, 8 * ev.shape[1], ev, det=False, jit=True)
    assert r0.tolist() == case["expect"]["r0"]


def test_divergent_loops_jit(ctx):
    lines = ["ldx8 r2 r1 0", "and r2 63", "mov r0 0", "jeq r2 0 done", "l:", "add r0 r2", "add r2 -1",
             "jne r2 0 l", "done:", "exit"]
    ev = np.zeros((5000, 2), dtype=np.uint64)
    ev[:, 0] = np.random.default_rng(2).integers(0, 1 << 40, 5000)
    _, _, r0, _ = run_both(ctx, assemble(lines).prog(), [], 16, ev, det=False, jit=True)
    k = (ev[:, 0] & 63).astype(np.int64)
    assert np.array_equal(r0, k * (k + 1) // 2)


def test_budget_trip_jit(ctx):
    import paper_2512_12615_gb300 as gx

    lines = ["mov r0 0", "mov r2 0", "l:", "add r0 1", "add r2 1", "jlt r2 5000 l", "exit"]
    p = gx.Program(ctx, assemble(lines).prog(), [], 16, insn_budget=100, jit=True)
    ev = np.zeros((77, 2), dtype=np.uint64)
    ret = torch.full((77,), 7, dtype=torch.int64, device="cuda")
    p.run(device_events(ev), 77, ret_out=ret)
    st = p.status(reset=True)
    assert st.status == gx.E_BUDGET and st.budget_trips == 77 and int(ret.abs().sum()) == 0


@pytest.mark.parametrize("insert_only", [False, True])
def test_page_heat_hash_flavours_two_launches(ctx, insert_only):
    """Ordered probes (ordinary hash map) and L1-first probes (insert-only map): the second
    launch finds every key published, the first one races inserts against lookups."""
    import paper_2512_12615_gb300 as gx
    import oracle as O
    from tests.parity import assert_same, gpu_maps, snapshot_gpu, snapshot_oracle

    prog, specs, cs = P.page_heat()
    specs = [dict(s) for s in specs]
    if insert_only:
        assert specs[0]["flags"] == gx.MAP_F_NO_DELETE
    else:
        specs[0].pop("flags", None)
    ev = gen.pageheat_events(150_001, seed=77)
    gm = gpu_maps(ctx, specs)
    p = gx.Program(ctx, prog, gm, cs, deterministic=True, jit=True)
    dev = device_events(ev)
    om = O.maps_from_specs(specs)
    for _ in range(2):
        p.run(dev, len(ev))
        O.run(prog, om, ev, cs)
    torch.cuda.synchronize()
    assert p.status().status == 0
    assert_same(snapshot_gpu(gm), snapshot_oracle(om))


def test_map_flags_are_checked(ctx):
    import paper_2512_12615_gb300 as gx

    with pytest.raises(gx.GxError):
        gx.Map(ctx, gx.MAP_ARRAY, 4, 8, 16, flags=gx.MAP_F_NO_DELETE)
    with pytest.raises(gx.GxError):
        gx.Map(ctx, gx.MAP_HASH, 8, 8, 16, flags=2)
    m = gx.Map(ctx, gx.MAP_HASH, 8, 8, 16, flags=gx.MAP_F_NO_DELETE)
    prog = assemble(["mov r6 r1", "ldx8 r7 r6 0", "stx8 r10 -8 r7", "ld_map r1 0", "mov r2 r10", "add r2 -8",
                     "call map_delete_elem", "mov r0 0", "exit"]).prog()
    with pytest.raises(gx.GxError):
        gx.Program(ctx, prog, [m], 16)
    m.destroy()


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_kernel_variants(ctx, variant):
    """The wide and the register-capped entry of a specialised program give the same results."""
    prog, specs, cs = P.page_heat()
    ev = gen.pageheat_events(100_003, seed=91)
    ev["size"][::97] = 3
    run_both(ctx, prog, specs, cs, ev, jit=True, launch=(256, 8, 0, variant))
    prog, specs, cs = P.latency(ring_bytes=1 << 22)
    run_both(ctx, prog, specs, cs, gen.latency_pairs(50_001, seed=92), jit=True, launch=(128, 4, 0, variant))
