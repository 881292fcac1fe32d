"""Block-scheduling hook policies (the `should_try_steal` hook of Sec. 4.3.2, the FixedWork /
Greedy / LatencyBudget schedulers of Sec. 6), host side: their decisions on the oracle
equal the closed forms; they are warp-uniform handlers within a hook budget, whose worst
paths are counted by hand; their statistics are order-independent (deterministic mode).
On the device they steer a batch's stealing mode (gx_batch_set_sched): its walk is pinned in
tests/test_host_steal.py, its kernel compiles in tests/test_jit_compile.py, and its GPU
parity tests (tests/test_gpu_sched.py) have not yet run.
"""
import numpy as np
import pytest

import oracle as O
from workloads import programs as P

gx = pytest.importorskip("paper_2512_12615_gb300")

# worst paths, counted along each listing: (instructions, helper calls, memory operations)
WORST = {"fixed": (16, 1, 4), "greedy": (19, 1, 5), "latency_budget": (22, 1, 7)}


def contexts(n, seed):
    rng = np.random.default_rng(seed)
    ctx = np.zeros(n, dtype=[("block", "<u4"), ("sm", "<u4"), ("done", "<u4"), ("left", "<u4"),
                             ("elapsed", "<u8"), ("budget", "<u8")])
    ctx["block"] = rng.integers(0, 1024, n)
    ctx["sm"] = rng.integers(0, 152, n)
    ctx["done"] = rng.integers(0, 100, n)
    ctx["left"] = np.where(rng.random(n) < 0.3, 0, rng.integers(1, 10, n))
    ctx["budget"] = 1_000_000
    ctx["elapsed"] = rng.integers(0, 2_000_000, n)
    ctx["elapsed"][::11] = 1_000_000  # exactly at the budget
    assert ctx.dtype.itemsize == P.SCHED_CTX
    return ctx


def closed_form(kind, ctx):
    if kind == "fixed":
        return np.zeros(len(ctx), dtype=np.int64)
    steal = ctx["left"] > 0
    if kind == "latency_budget":
        steal &= ctx["elapsed"] < ctx["budget"]
    return steal.astype(np.int64)


@pytest.mark.parametrize("kind", sorted(WORST))
def test_decisions_and_statistics(kind):
    prog, specs, cs = P.sched_policy(kind)
    ctx = contexts(5_000, seed=len(kind))
    maps = O.maps_from_specs(specs)
    r0, _ = O.run(prog, maps, ctx, cs, want_r0=True)
    want = closed_form(kind, ctx)
    assert np.array_equal(r0, want)
    stats = maps[0].array_u64()
    grp = (ctx["sm"] & 7).astype(np.int64)
    assert np.array_equal(stats[:, 0], np.bincount(grp, minlength=P.SCHED_STATS))
    assert np.array_equal(stats[:, 1], np.bincount(grp, weights=want, minlength=P.SCHED_STATS).astype(np.uint64))


@pytest.mark.parametrize("kind", sorted(WORST))
def test_uniform_handler_within_a_hook_budget(kind):
    """Every field is the same for the block's threads; the worst path fits a hook budget of
    24 instructions, 1 helper call and 8 memory operations, and one instruction less than
    the worst path is refused."""
    prog, specs, cs = P.sched_policy(kind)
    uni = np.ones(cs, bool)
    rc, rep, log = gx.verify_simt(prog, specs, cs, uni, max_insns=24, max_helper_calls=1, max_mem_ops=8,
                                  deterministic=True)
    assert rc == 0, log
    assert (rep.max_insns, rep.max_helper_calls, rep.max_mem_ops) == WORST[kind]
    assert rep.varying_insns == 0
    rc, rep, _ = gx.verify_simt(prog, specs, cs, uni, max_insns=WORST[kind][0] - 1)
    assert rc == gx.E_VERIFY and rep.violation == gx.SIMT_V_INSNS
    rc, rep, _ = gx.verify_simt(prog, specs, cs, uni, max_mem_ops=WORST[kind][2] - 1)
    assert rc == gx.E_VERIFY and rep.violation == gx.SIMT_V_MEM


def test_oracle_max_path_is_the_counted_one():
    """A context on LatencyBudget's worst path (units left, under budget) runs exactly the
    22 instructions counted."""
    prog, specs, cs = P.sched_policy("latency_budget")
    ctx = contexts(1, seed=0)
    ctx["left"], ctx["elapsed"], ctx["budget"] = 3, 10, 1_000_000
    _, count = O.run(prog, O.maps_from_specs(specs), ctx, cs)
    assert count == WORST["latency_budget"][0]


def test_context_layout_is_the_engines():
    """The policies read the fields where the engine's stealing kernel writes them."""
    assert P.SCHED_CTX == gx.SCHED_CTX
    assert (P.SCHED_BLOCK, P.SCHED_SM, P.SCHED_DONE, P.SCHED_LEFT, P.SCHED_ELAPSED, P.SCHED_BUDGET) == (
        gx.SCHED_OFF_BLOCK, gx.SCHED_OFF_SM, gx.SCHED_OFF_DONE, gx.SCHED_OFF_LEFT, gx.SCHED_OFF_ELAPSED,
        gx.SCHED_OFF_BUDGET)
    # the default hook budget holds all three policies
    for kind in WORST:
        assert all(w <= m for w, m in zip(WORST[kind], (gx.SCHED_MAX_INSNS, gx.SCHED_MAX_HELPERS, gx.SCHED_MAX_MEM)))
