"""The work-stealing batch kernel (gx_batch_set_sched): a batch's blocks own contiguous
shares of the chunk table and a `should_try_steal` program (FixedWork, Greedy,
LatencyBudget; Sec. 4.3.2, Sec. 6) decides, before each chunk a block would take from
another share, whether it takes it.

What they hold it to:
  - the items' maps and R0 equal the oracle's, whatever the policy (every chunk runs once);
  - the per-block tallies: owned + stolen summed = the chunk count; FixedWork, and
    LatencyBudget with a zero budget, leave each block exactly its share;
  - the scheduling program's own statistics map counts exactly the asks and grants the
    tallies report (its decisions are per-SM-group counts, Sec. 6's policies as written);
  - the refusals: a scheduling program that is interpreted, warp-level, of another context
    size or over the hook budget; a batch with an interpreted item;
  - the same with one block per chunk and cluster launch control (launch_control=True):
    cancelled blocks leave zero rows, every other block ran its own chunk.
The walk itself (exactly-once under any interleaving) is pinned on the host
(tests/test_host_steal.py); the kernel compiles on the host (tests/test_jit_compile.py).
The `first_run` cases are the smallest: one small item, FixedWork (then Greedy under launch
control, the first use of its cancel and bounded mbarrier wait).
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

PICK = [0, 5, 11, 19, 27, 33, 48, 63]
SIZES = [5000, 77, 20011, 1, 33333, 4096, 12345, 9999]


@pytest.fixture(scope="module")
def ctx():
    return gx.Context(0)


def hook_program(ctx, kind):
    hook, hook_specs, cs = P.sched_policy(kind)
    hm = gpu_maps(ctx, hook_specs)
    return gx.Program(ctx, hook, hm, cs, jit=True), hm


def make_items(ctx, picks, sizes, seed):
    progs = P.batch_programs()
    items = []
    for k, (p, n) in enumerate(zip(picks, sizes)):
        prog, specs, cs = progs[p]
        ev = gen.uniform_events(n, seed=seed + k)
        gm = gpu_maps(ctx, specs)
        items.append(dict(prog=prog, specs=specs, cs=cs, ev=ev, dev=device_events(ev), gm=gm,
                          gp=gx.Program(ctx, prog, gm, cs, deterministic=True, jit=True),
                          ret=torch.zeros(n, dtype=torch.int64, device="cuda")))
    return items


def share_sizes(nchunks, shares):
    lo = [s * nchunks // shares for s in range(shares + 1)]
    return np.diff(np.array(lo, dtype=np.int64))


def run_sched(ctx, items, kind, budget_ns, shape, launches=1, launch_control=False):
    hp, hm = hook_program(ctx, kind)
    b = gx.Batch(ctx)
    for it in items:
        b.add(it["gp"], it["dev"], len(it["ev"]), it["ret"])
    b.set_sched(hp, budget_ns, launch_control=launch_control)
    b.plan(launch=shape)
    tallies = []
    for _ in range(launches):
        b.launch()
        tallies.append(b.sched_tally())
    torch.cuda.synchronize()
    stats = hm[0].array_u64()
    status = hp.status().status
    b.destroy()
    return tallies, stats, status


def check_items(items, repeats):
    for it in items:
        om = O.maps_from_specs(it["specs"])
        for _ in range(repeats):
            r0, _ = O.run(it["prog"], om, it["ev"], it["cs"], want_r0=True)
        assert np.array_equal(it["ret"].cpu().numpy(), r0)
        assert_same(snapshot_gpu(it["gm"]), snapshot_oracle(om))
        assert it["gp"].status().status == 0


def check_tally(t, nchunks, never_steals):
    own, stolen, asked, granted = (t[:, k].astype(np.int64) for k in range(gx.STEAL_WORDS))
    assert int(own.sum() + stolen.sum()) == nchunks
    assert (asked >= granted).all() and (granted >= stolen).all()
    assert (granted - stolen <= len(t) - 1).all()
    if never_steals:
        assert np.array_equal(own, share_sizes(nchunks, len(t)))
        assert stolen.sum() == 0 and granted.sum() == 0
        assert (asked <= 1).all()


def test_first_run_fixed_small(ctx):
    """One item of 5000 events in 256 x 4 chunks (5 chunks), FixedWork: no block steals."""
    items = make_items(ctx, [0], [5000], seed=100)
    (t,), stats, status = run_sched(ctx, items, "fixed", 0, (256, 4))
    assert status == 0
    check_items(items, 1)
    check_tally(t, 5, never_steals=True)
    assert int(stats[:, 0].sum()) == int(t[:, gx.STEAL_ASKED].sum())
    assert int(stats[:, 1].sum()) == 0


@pytest.mark.parametrize("kind,budget_ns", [("fixed", 0), ("greedy", 0), ("latency_budget", 0),
                                            ("latency_budget", 10**12)])
@pytest.mark.parametrize("shape", [(256, 4), (128, 1)])
def test_policies_match_oracle(ctx, kind, budget_ns, shape):
    items = make_items(ctx, PICK, SIZES, seed=200)
    tallies, stats, status = run_sched(ctx, items, kind, budget_ns, shape, launches=2)
    assert status == 0
    check_items(items, 2)  # a relaunch replays the graph: maps accumulate, R0 is rewritten
    ce = shape[0] * shape[1]
    nchunks = sum((n + ce - 1) // ce for n in SIZES)
    never = kind == "fixed" or (kind == "latency_budget" and budget_ns == 0)
    for t in tallies:
        check_tally(t, nchunks, never)
    # the scheduling program counted every ask and every grant of both launches
    assert int(stats[:, 0].sum()) == int(sum(t[:, gx.STEAL_ASKED].sum() for t in tallies))
    assert int(stats[:, 1].sum()) == int(sum(t[:, gx.STEAL_GRANTED].sum() for t in tallies))


def check_tally_lc(t, nchunks, never_steals):
    """One block per chunk: rows of cancelled blocks are zero, every other block ran its own
    chunk, and one failed cancel at most ends each walk."""
    own, stolen, asked, granted = (t[:, k].astype(np.int64) for k in range(gx.STEAL_WORDS))
    assert len(t) == max(nchunks, 1)
    assert int(own.sum() + stolen.sum()) == nchunks
    assert set(own.tolist()) <= {0, 1}
    assert (asked >= granted).all() and (granted >= stolen).all() and (granted - stolen <= 1).all()
    assert int(own.sum()) == nchunks - int(stolen.sum())  # a block is cancelled or runs its own chunk
    if never_steals:
        assert (own == 1).all() and stolen.sum() == 0 and granted.sum() == 0


def test_first_run_launch_control_small(ctx):
    """Cluster launch control, smallest case: 5 chunks, one block each, FixedWork (no cancel
    is ever issued).  Then Greedy on the same sizes, where blocks may cancel."""
    items = make_items(ctx, [0], [5000], seed=110)
    (t,), stats, status = run_sched(ctx, items, "fixed", 0, (256, 4), launch_control=True)
    assert status == 0
    check_items(items, 1)
    check_tally_lc(t, 5, never_steals=True)
    items = make_items(ctx, [0], [5000], seed=111)
    (t,), stats, status = run_sched(ctx, items, "greedy", 0, (256, 4), launch_control=True)
    assert status == 0
    check_items(items, 1)
    check_tally_lc(t, 5, never_steals=False)
    assert int(stats[:, 1].sum()) == int(t[:, gx.STEAL_GRANTED].sum())


@pytest.mark.parametrize("kind,budget_ns", [("fixed", 0), ("greedy", 0), ("latency_budget", 10**12)])
def test_launch_control_matches_oracle(ctx, kind, budget_ns):
    items = make_items(ctx, PICK, SIZES, seed=500)
    tallies, stats, status = run_sched(ctx, items, kind, budget_ns, (256, 4), launches=2, launch_control=True)
    assert status == 0
    check_items(items, 2)
    nchunks = sum((n + 1023) // 1024 for n in SIZES)
    for t in tallies:
        check_tally_lc(t, nchunks, kind == "fixed")
    assert int(stats[:, 0].sum()) == int(sum(t[:, gx.STEAL_ASKED].sum() for t in tallies))
    assert int(stats[:, 1].sum()) == int(sum(t[:, gx.STEAL_GRANTED].sum() for t in tallies))


def test_greedy_steals_under_imbalance(ctx):
    """The heaviest generated program over many events next to light ones: the blocks that
    own light chunks finish first and take heavy ones.  (Stealing depends on timing; with
    this imbalance a run without a single steal would mean the hook is never granted.)"""
    progs = P.batch_programs()
    heavy = max(range(len(progs)), key=lambda p: len(progs[p][0]))
    items = make_items(ctx, [heavy] + PICK[:4], [1 << 20, 4096, 4096, 4096, 4096], seed=300)
    (t,), _, status = run_sched(ctx, items, "greedy", 0, (256, 4))
    assert status == 0
    check_items(items, 1)
    nchunks = sum((len(it["ev"]) + 1023) // 1024 for it in items)
    check_tally(t, nchunks, never_steals=False)
    assert t[:, gx.STEAL_STOLEN].sum() > 0


def test_refusals(ctx):
    items = make_items(ctx, [0], [100], seed=400)
    hook, hook_specs, cs = P.sched_policy("greedy")
    hm = gpu_maps(ctx, hook_specs)
    b = gx.Batch(ctx)
    b.add(items[0]["gp"], items[0]["dev"], 100, items[0]["ret"])
    with pytest.raises(gx.GxError) as e:  # interpreted: the stealing kernel exists only as specialised code
        b.set_sched(gx.Program(ctx, hook, hm, cs), 0)
    assert e.value.status == gx.EINVAL
    with pytest.raises(gx.GxError) as e:  # the warp-level form: the hook runs on one lane
        b.set_sched(gx.Program(ctx, hook, hm, cs, jit=True, simt={"uniform": np.ones(cs, bool)}), 0)
    assert e.value.status == gx.EINVAL
    with pytest.raises(gx.GxError) as e:  # over a hook budget of 10 instructions
        b.set_sched(gx.Program(ctx, hook, hm, cs, jit=True), 0, max_insns=10)
    assert e.value.status == gx.E_VERIFY
    with pytest.raises(gx.GxError) as e:  # not a GX_SCHED_CTX-byte context
        b.set_sched(gx.Program(ctx, assemble(["mov r0 1", "exit"]).prog(), [], 16, jit=True), 0)
    assert e.value.status == gx.EINVAL
    with pytest.raises(gx.GxError) as e:  # no scheduling program yet
        b.sched_tally()
    assert e.value.status == gx.EINVAL
    b.destroy()
    # an interpreted item: the batch cannot build the stealing kernel
    gm = gpu_maps(ctx, items[0]["specs"])
    interp = gx.Program(ctx, items[0]["prog"], gm, items[0]["cs"], deterministic=True)
    b = gx.Batch(ctx)
    b.add(interp, items[0]["dev"], 100, None)
    b.set_sched(gx.Program(ctx, hook, hm, cs, jit=True), 0)
    with pytest.raises(gx.GxError) as e:
        b.plan(launch=(256, 4))
    assert e.value.status == gx.EINVAL
    b.destroy()


def test_scheduling_program_ring_records(ctx):
    """A scheduling program that writes its context's first word (block | SM << 32) to a ring
    buffer at every ask and steals while chunks are left: one record per ask, each carrying
    its block index as the event index (the gx_batch_set_sched contract)."""
    lines = ["mov r6 r1", "ldx8 r7 r6 0", "stx8 r10 -8 r7", "ld_map r1 0", "mov r2 r10", "add r2 -8", "mov r3 8",
             "mov r4 0", "call ringbuf_output", "ldx4 r0 r6 12", "exit"]
    ring_spec = [dict(type=gx.MAP_RINGBUF, key_size=0, value_size=0, max_entries=1 << 20)]
    ring = gpu_maps(ctx, ring_spec)
    hp = gx.Program(ctx, assemble(lines).prog(), ring, gx.SCHED_CTX, jit=True)
    items = make_items(ctx, PICK, SIZES, seed=600)
    b = gx.Batch(ctx)
    for it in items:
        b.add(it["gp"], it["dev"], len(it["ev"]), it["ret"])
    b.set_sched(hp, 0)
    b.plan(launch=(128, 1))
    b.launch()
    t = b.sched_tally()
    torch.cuda.synchronize()
    raw, dropped = ring[0].drain()
    recs = gx.parse_records(raw)
    assert dropped == 0 and len(recs) == int(t[:, gx.STEAL_ASKED].sum())
    for idx, payload in recs:
        word = int.from_bytes(payload, "little")
        assert idx == (word & 0xFFFFFFFF) < len(t)
    check_items(items, 1)
    b.destroy()
