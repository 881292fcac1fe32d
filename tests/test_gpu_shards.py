"""Block-private combining of map updates (the hierarchical maps of Sec. 5.3) against the
oracle, bit for bit: every update kind at every map-sharding width, the carry of 64-bit
adds split into 32-bit halves, identities of AND / MIN over non-zero initial values,
caches small enough that most updates miss, and the persistent (batched) kernel."""
import numpy as np
import pytest

import oracle as O
from tests.asmtext import assemble
from tests.parity import assert_same, device_events, gpu_maps, run_both, snapshot_gpu, snapshot_oracle
from workloads import gen
from workloads import programs as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

OFF = 255
AGG = 0x100

# array map 0: 8 values of 64 bytes, one update kind per word; hash map 1: 64 keys, same layout
ALLOPS = """
mov r6 r1
ldx8 r7 r6 0
ldx8 r8 r6 8
ldx8 r9 r6 24
and r9 7
stx4 r10 -4 r9
ld_map r1 0
mov r2 r10
add r2 -4
call map_lookup_elem
jeq r0 0 hash
mov r9 r0
mov r1 r7
atomic8 add r0 0 r1
mov r1 r8
atomic4 add r0 8 r1
mov r1 r7
atomic8 or r0 16 r1
mov r1 r8
and r1 0xFFF
jne r1 0 keep
mov r2 r7
and r2 63
mov r1 1
lsh r1 r2
xor r1 -1
atomic8 and r0 24 r1
keep:
mov r1 r8
atomic8 xor r0 32 r1
mov r1 r9
add r1 40
mov r2 r7
call atomic_max_u64
mov r1 r9
add r1 48
mov r2 r8
call atomic_min_u64
mov r0 r9
mov r1 r7
atomic4 or r0 56 r1
mov r1 r8
atomic4 xor r0 60 r1
hash:
mov r1 r7
rsh r1 58
stx8 r10 -8 r1
ld_map r1 1
mov r2 r10
add r2 -8
call map_lookup_elem
jne r0 0 have
st8 r10 -72 0
st8 r10 -64 0
st8 r10 -56 0
st8 r10 -48 0
st8 r10 -40 0
st8 r10 -32 0
st8 r10 -24 0
st8 r10 -16 0
ld_map r1 1
mov r2 r10
add r2 -8
mov r3 r10
add r3 -72
mov r4 1
call map_update_elem
ld_map r1 1
mov r2 r10
add r2 -8
call map_lookup_elem
jeq r0 0 out
have:
mov r9 r0
mov r1 r8
atomic8 add r0 0 r1
mov r1 r7
atomic4 add r0 8 r1
mov r1 r8
atomic8 or r0 16 r1
mov r1 r7
atomic8 xor r0 32 r1
mov r1 r9
add r1 40
mov r2 r8
call atomic_max_u64
mov r0 r9
mov r1 r8
atomic4 xor r0 60 r1
out:
mov r0 0
exit
""".strip().splitlines()

SPECS = [dict(type=2, key_size=4, value_size=64, max_entries=8), dict(type=1, key_size=8, value_size=64, max_entries=128)]


def allops_events(n, seed):
    ev = np.random.default_rng(seed).integers(0, 2**64 - 1, size=(n, 4), dtype=np.uint64, endpoint=True)
    return ev


def allops_init():
    v = np.zeros((8, 8), dtype=np.uint64)
    v[:, 3] = np.uint64(2**64 - 1)  # AND word starts all ones
    v[:, 6] = np.uint64(2**64 - 1)  # MIN word starts at the maximum
    v[:, 0] = np.uint64(2**64 - 5)  # ADD word near the wrap
    return [v.tobytes(), None]


@pytest.fixture(scope="module")
def ctx():
    import paper_2512_12615_gb300 as gx

    return gx.Context(0)


def test_allops_is_combinable():
    import paper_2512_12615_gb300 as gx

    rc, info, log = gx.analyze(assemble(ALLOPS).prog(), SPECS, 32, deterministic=True)
    assert rc == 0, log
    assert info.combinable_maps == 3


@pytest.mark.parametrize("shards", [OFF, 2, 3, 0, 10, 2 | AGG, AGG])
@pytest.mark.parametrize("shape", [(64, 3), (256, 8)])
def test_allops_every_width(ctx, shards, shape):
    ev = allops_events(50_003, seed=7 + shards)
    run_both(ctx, assemble(ALLOPS).prog(), SPECS, 32, ev, jit=True, launch=shape + (shards,), init=allops_init())


def test_allops_tiny_batch(ctx):
    for n in (1, 31, 33):
        run_both(ctx, assemble(ALLOPS).prog(), SPECS, 32, allops_events(n, seed=n), jit=True, launch=(256, 4, 0),
                 init=allops_init())


@pytest.mark.parametrize("shards", [OFF, 2, 0, 2 | AGG])
def test_page_heat_widths(ctx, shards):
    prog, specs, cs = P.page_heat()
    ev = gen.pageheat_events(300_007, seed=41)
    ev["size"][::97] = 3
    ev["kind"][5::101] = 9
    ev["addr"][7::89] |= np.uint64(1)
    run_both(ctx, prog, specs, cs, ev, jit=True, launch=(256, 8, shards))


@pytest.mark.parametrize("shards", [OFF, 4, 0])
def test_counting_and_latency_widths(ctx, shards):
    prog, specs, cs = P.counting()
    run_both(ctx, prog, specs, cs, gen.uniform_events(100_003, seed=42), jit=True, launch=(128, 4, shards))
    prog, specs, cs = P.latency(ring_bytes=1 << 22)
    run_both(ctx, prog, specs, cs, gen.latency_pairs(60_001, seed=43), jit=True, launch=(256, 2, shards))


@pytest.mark.parametrize("p", [1, 8, 22, 40, 57])
@pytest.mark.parametrize("agg", [0, AGG])
def test_random_programs_narrow_cache(ctx, p, agg):
    prog, specs, cs = P.batch_programs()[p]
    run_both(ctx, prog, specs, cs, gen.uniform_events(30_011, seed=500 + p), jit=True, launch=(256, 4, 2 | agg))


@pytest.mark.parametrize("shards", [OFF, 3, 0, 3 | AGG])
def test_batch_kernel_with_shards(ctx, shards):
    """The persistent multi-program kernel flushes each chunk's combined updates."""
    import paper_2512_12615_gb300 as gx

    cases = [(assemble(ALLOPS).prog(), SPECS, 32, allops_events(40_000, seed=9)),
             P.page_heat() + (gen.pageheat_events(70_001, seed=10),),
             P.counting() + (gen.uniform_events(9_999, seed=11),)]
    items = []
    b = gx.Batch(ctx)
    for prog, specs, cs, ev in cases:
        gm = gpu_maps(ctx, specs)
        gp = gx.Program(ctx, prog, gm, cs, deterministic=True, jit=True)
        dev = device_events(ev)
        ret = torch.zeros(len(ev), dtype=torch.int64, device="cuda")
        b.add(gp, dev, len(ev), ret)
        items.append((prog, specs, cs, ev, gm, gp, dev, ret))
    b.plan(launch=(256, 4, shards))
    b.launch()
    b.launch()
    torch.cuda.synchronize()
    for prog, specs, cs, ev, gm, gp, dev, ret in items:
        om = O.maps_from_specs(specs)
        for _ in range(2):
            r0, _ = O.run(prog, om, ev, cs, want_r0=True)
        assert np.array_equal(ret.cpu().numpy(), r0)
        assert_same(snapshot_gpu(gm), snapshot_oracle(om))
        assert gp.status().status == 0
    b.destroy()


def test_autotune_reports_a_width(ctx):
    import paper_2512_12615_gb300 as gx

    prog, specs, cs = P.page_heat()
    ev = gen.pageheat_events(1 << 20, seed=12)
    gm = gpu_maps(ctx, specs)
    p = gx.Program(ctx, prog, gm, cs, deterministic=True, jit=True)
    block, ept, shards = p.autotune(device_events(ev), len(ev))
    assert block in (128, 256) and 1 <= ept <= 64 and shards in (0, AGG, OFF, 10)
    # tuning ran on scratch copies: the real maps are untouched
    assert len(gm[0].hash_items()) == 0 and not gm[1].array_values().any()


@pytest.mark.parametrize("shards", [0, 10, 4 | AGG])
def test_three_caches_and_a_copy(ctx, shards):
    """Four combinable maps in one program: a private array copy and three caches whose offsets
    depend on the launch's width (the widest narrowed so that the area fits)."""
    from tests.test_jit_compile import MANY, MANY_SPECS

    ev = np.random.default_rng(5).integers(0, 2**63, size=(40_009, 4), dtype=np.uint64)
    run_both(ctx, assemble(MANY).prog(), MANY_SPECS, 32, ev, jit=True, launch=(256, 4, shards))
