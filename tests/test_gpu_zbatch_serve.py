"""Batched (one persistent kernel from a captured graph) and served (continuous batching)
forms against the oracle and against plain per-request launches."""
import numpy as np
import pytest

import oracle as O
from tests.parity import assert_same, device_events, gpu_maps, snapshot_gpu, snapshot_oracle
from workloads import gen
from workloads import programs as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PICK = [0, 5, 11, 19, 27, 33, 48, 63]
SIZES = [5000, 77, 20011, 1, 33333, 4096, 12345, 9999]


@pytest.fixture(scope="module")
def ctx():
    import paper_2512_12615_gb300 as gx

    return gx.Context(0)


def make_items(ctx, jit, seed=0):
    import paper_2512_12615_gb300 as gx

    progs = P.batch_programs()
    items = []
    for k, (p, n) in enumerate(zip(PICK, SIZES)):
        prog, specs, cs = progs[p]
        ev = gen.uniform_events(n, seed=seed + 1000 + k)
        gm = gpu_maps(ctx, specs)
        items.append(dict(prog=prog, specs=specs, cs=cs, ev=ev, dev=device_events(ev), gm=gm,
                          gp=gx.Program(ctx, prog, gm, cs, deterministic=True, jit=jit),
                          ret=torch.zeros(n, dtype=torch.int64, device="cuda")))
    return items


def oracle_of(items, repeats=1):
    out = []
    for it in items:
        om = O.maps_from_specs(it["specs"])
        for _ in range(repeats):
            r0, _ = O.run(it["prog"], om, it["ev"], it["cs"], want_r0=True)
        out.append((om, r0))
    return out


@pytest.mark.parametrize("jit", [False, True])
@pytest.mark.parametrize("shape", [(256, 4), (128, 1), None])
def test_batch_matches_oracle(ctx, jit, shape):
    import paper_2512_12615_gb300 as gx

    items = make_items(ctx, jit)
    b = gx.Batch(ctx)
    for it in items:
        b.add(it["gp"], it["dev"], len(it["ev"]), it["ret"])
    b.plan(launch=shape)  # None: autotuned on scratch copies of the maps
    b.launch()
    b.launch()  # a relaunch replays the graph: maps accumulate, R0 is rewritten
    torch.cuda.synchronize()
    for it, (om, r0) in zip(items, oracle_of(items, repeats=2)):
        assert np.array_equal(it["ret"].cpu().numpy(), r0)
        assert_same(snapshot_gpu(it["gm"]), snapshot_oracle(om))
        assert it["gp"].status().status == 0
    b.destroy()


@pytest.mark.parametrize("mode", ["batched", "batched_jit", "plain"])
def test_server_results_alone_equal_mix(ctx, mode):
    """Each request's R0 is the same run alone (plain launch) and inside the served mix;
    the resident maps end equal to the oracle over all requests."""
    import paper_2512_12615_gb300 as gx

    items = make_items(ctx, mode == "batched_jit", seed=7)
    alone = []
    for it in items:  # alone: one plain launch per request on fresh maps
        gm = gpu_maps(ctx, it["specs"])
        p = gx.Program(ctx, it["prog"], gm, it["cs"], deterministic=True)
        r = torch.zeros(len(it["ev"]), dtype=torch.int64, device="cuda")
        p.run(it["dev"], len(it["ev"]), ret_out=r)
        alone.append(r.cpu().numpy())
    progs = [it["gp"] for it in items] if mode == "batched_jit" else []
    srv = gx.Server(ctx, mem_budget=1 << 30, max_inflight=3, max_items=64, plain=(mode == "plain"), progs=progs)
    reqs = []
    for rep in range(3):  # every program three times, interleaved
        for k, it in enumerate(items):
            reqs.append((it["gp"], it["dev"], len(it["ev"]), it["ret"] if rep == 2 else None, rep * 100 + k,
                         0.0002 * len(reqs)))
    srv.replay(reqs)
    done = []
    while len(done) < len(reqs):
        got = srv.poll(256, wait_ms=2000)
        assert got, "server made no progress"
        done += got
    assert all(c.status == 0 for c in done)
    assert sorted(c.tag for c in done) == sorted(r[4] for r in reqs)
    assert all(c.t_done >= c.t_start >= c.t_arrival - 1e-3 for c in done)
    srv.destroy()
    torch.cuda.synchronize()
    for it, a, (om, r0) in zip(items, alone, oracle_of(items, repeats=3)):
        assert np.array_equal(it["ret"].cpu().numpy(), a)
        assert np.array_equal(a, r0)
        assert_same(snapshot_gpu(it["gm"]), snapshot_oracle(om))


def test_server_admission_budget(ctx):
    import paper_2512_12615_gb300 as gx

    items = make_items(ctx, False, seed=9)
    srv = gx.Server(ctx, mem_budget=4 << 20, max_inflight=2)
    big = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(gx.GxError) as e:
        srv.submit(items[0]["gp"], big, (4 << 20) // 32 + (1 << 17))  # events alone exceed the budget
    assert e.value.status == gx.E_ADMISSION
    srv.submit(items[1]["gp"], items[1]["dev"], len(items[1]["ev"]), tag=5)
    got = []
    while not got:
        got = srv.poll(8, wait_ms=2000)
    assert got[0].tag == 5 and got[0].status == 0
    srv.destroy()
