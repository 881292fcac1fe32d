"""The warp-level form (gx_verify_load_simt) against the oracle's warp run, bit for bit.

They cover warp_heat over warp-context records with planted bad warps, misaligned lanes
and a ragged last warp; random SIMT handlers accepted in deterministic mode; one warp of
the program with every shared effect; several launch shapes and combining widths; and
the refusals (no interpreter form; a batch that would interpret it).

The generated form puts leader-only code (helper calls with bounded probe loops) inside
`if (lead)`, then joins the warp's valid lanes with __syncwarp and broadcasts.  Every lane
of that mask reaches every join: the mask is taken at entry, SIMT verification makes each
branch uniform across the valid lanes, and exits and budget trips are uniform too.  The
`first_run` cases are the smallest (one warp), for a first run on new hardware.
"""
import numpy as np
import pytest

import oracle as O
from tests.asmtext import assemble
from workloads import gen
from workloads import programs as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2512_12615_gb300 as gx  # noqa: E402
from tests.parity import assert_same, device_events, gpu_maps, snapshot_gpu, snapshot_oracle  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    return gx.Context(0)


def run_warp_both(ctx, prog, specs, cs, ev, uniform, launch=None):
    """The engine's warp-level form and the oracle's warp run over the same records:
    maps, ring records and R0 per record must be equal."""
    gm = gpu_maps(ctx, specs)
    p = gx.Program(ctx, prog, gm, cs, jit=True, simt={"uniform": uniform})
    raw = np.ascontiguousarray(ev).view(np.uint8).reshape(-1, cs)
    n = raw.shape[0]
    ret = torch.full((n,), -7, dtype=torch.int64, device="cuda")
    p.run(device_events(raw), n, ret_out=ret, launch=launch)
    torch.cuda.synchronize()
    assert p.status().status == 0
    om = O.maps_from_specs(specs)
    r0, _ = O.run_warps(prog, om, raw, cs, uniform=uniform, want_r0=True)
    assert np.array_equal(ret.cpu().numpy(), r0)
    assert_same(snapshot_gpu(gm), snapshot_oracle(om))
    p.destroy()


def test_first_run_reduction_only(ctx):
    """The smallest case, to run first: one warp, a warp reduction, no leader block."""
    ev = np.zeros((32, 2), dtype=np.uint64)
    ev[:, 1] = np.arange(32, dtype=np.uint64) * np.uint64(3)
    prog = assemble(["ldx8 r1 r1 8", "call warp_sum_u64", "exit"]).prog()
    run_warp_both(ctx, prog, [], 16, ev, [True] * 8 + [False] * 8, launch=(64, 1))


def test_first_run_one_leader_block(ctx):
    """Next: one leader block (a lookup), then the barrier and the broadcast."""
    ev = np.zeros((32, 2), dtype=np.uint64)
    ev[:, 1] = np.arange(32, dtype=np.uint64)
    lines = ["ldx8 r7 r1 0", "stx4 r10 -4 r7", "ld_map r1 0", "mov r2 r10", "add r2 -4", "call map_lookup_elem",
             "mov r6 0", "jeq r0 0 out", "mov r6 1", "out:", "mov r0 r6", "exit"]
    specs = [dict(type=2, key_size=4, value_size=8, max_entries=4)]
    run_warp_both(ctx, assemble(lines).prog(), specs, 16, ev, [True] * 8 + [False] * 8, launch=(64, 1))


@pytest.mark.parametrize("launch", [None, (64, 1), (256, 8, 255), (256, 4, 0), (128, 2, 4)])
def test_warp_heat(ctx, launch):
    from tests.test_oracle_closed_forms import warp_heat_events

    prog, specs, cs = P.warp_heat()
    run_warp_both(ctx, prog, specs, cs, warp_heat_events(3_000, seed=31), gen.WARP_UNIFORM, launch)


def test_random_handlers(ctx):
    from tests.test_simt_verifier import RANDOM_SPECS, random_handler, random_warps

    rng = np.random.default_rng(91)
    done = 0
    while done < 12:
        lines = random_handler(rng)
        words = rng.random(4) < 0.5
        uniform = np.repeat(words, 8)
        prog = assemble(lines).prog()
        if gx.verify_simt(prog, RANDOM_SPECS, 32, uniform, deterministic=True)[0] != 0:
            continue
        run_warp_both(ctx, prog, RANDOM_SPECS, 32, random_warps(rng, words, warps=40), uniform)
        done += 1


@pytest.mark.parametrize("n", [32, 13])
def test_every_shared_effect_in_one_warp(ctx, n):
    """Exchanges and plain stores are order-dependent across warps; one warp fixes the order."""
    from tests.test_jit_compile import EVERY_EFFECT, EVERY_EFFECT_SPECS, WARP_UNI
    from tests.test_simt_verifier import random_warps

    ev = random_warps(np.random.default_rng(n), [False, True, True, True], warps=1, tail=0)[:n]
    run_warp_both(ctx, assemble(EVERY_EFFECT).prog(), EVERY_EFFECT_SPECS, 32, ev, WARP_UNI)


def test_refusals(ctx):
    prog, specs, cs = P.warp_heat()
    gm = gpu_maps(ctx, specs)
    with pytest.raises(gx.GxError) as e:
        gx.Program(ctx, prog, gm, cs, jit=False, simt={"uniform": gen.WARP_UNIFORM})
    assert e.value.status == gx.EINVAL
    warp = gx.Program(ctx, prog, gm, cs, jit=True, simt={"uniform": gen.WARP_UNIFORM})
    cprog, cspecs, ccs = P.counting()
    plain = gx.Program(ctx, cprog, gpu_maps(ctx, cspecs), ccs)  # interpreted
    b = gx.Batch(ctx)
    ev = device_events(gen.warp_access_events(4, seed=1))
    b.add(warp, ev, 128, None)
    b.add(plain, device_events(gen.uniform_events(64, seed=2)), 64, None)
    with pytest.raises(gx.GxError) as e:
        b.plan()
    assert e.value.status == gx.EINVAL
    b.destroy()
