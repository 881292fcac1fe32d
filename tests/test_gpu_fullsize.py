"""Full-size results on the GPU, bit-exact, at the sizes the benchmark streams.

Page-heat and latency at 16M records against their closed forms (tests/closed_forms.py),
in the autotuned launch configuration the benchmark times; the 64-program batch at its
generated sizes (172M events) in one persistent launch against the oracle, program by
program (the oracle runs on every host core, one program per thread).
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O
from tests import closed_forms as CF
from tests.parity import assert_same, snapshot_gpu, snapshot_oracle
from workloads import gen
from workloads import programs as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N16M = 16 << 20


@pytest.fixture(scope="module")
def ctx():
    import paper_2512_12615_gb300 as gx

    return gx.Context(0)


def _dev(ev):
    return torch.from_numpy(np.ascontiguousarray(ev).view(np.uint8).reshape(-1)).cuda()


@pytest.mark.parametrize("jit", [True, False])
def test_page_heat_16M(ctx, jit):
    import paper_2512_12615_gb300 as gx

    prog, specs, cs = P.page_heat()
    ev = gen.pageheat_events(N16M, seed=0x6758 ^ 0x16)
    dev = _dev(ev)
    maps = [gx.Map.from_spec(ctx, s) for s in specs]
    p = gx.Program(ctx, prog, maps, cs, deterministic=True, jit=jit)
    p.autotune(dev, N16M)
    p.run(dev, N16M)
    p.run(dev, N16M)
    torch.cuda.synchronize()
    assert p.status().status == 0
    heat, tally = CF.page_heat(ev)
    got = maps[0].hash_items()
    assert len(got) == len(heat)
    for k, (c, t) in heat.items():
        v = got[int(k).to_bytes(8, "little")]
        assert (int.from_bytes(v[:8], "little"), int.from_bytes(v[8:], "little")) == (2 * c, t), k
    assert np.array_equal(maps[1].array_u64(), tally * np.uint64(2))
    p.destroy()
    for m in maps:
        m.destroy()


@pytest.mark.parametrize("jit", [True, False])
def test_latency_16M_records(ctx, jit):
    import paper_2512_12615_gb300 as gx

    prog, specs, cs = P.latency()
    pairs = N16M // 2
    ev = gen.latency_pairs(pairs, seed=0x6758 ^ 0x17)
    dev = _dev(ev)
    maps = [gx.Map.from_spec(ctx, s) for s in specs]
    p = gx.Program(ctx, prog, maps, cs, deterministic=True, jit=jit)
    p.autotune(dev, pairs)
    maps[1].drain()
    p.run(dev, pairs)
    torch.cuda.synchronize()
    assert p.status().status == 0
    hist, sel, recs = CF.latency_arrays(ev)
    assert np.array_equal(maps[0].array_u64()[:, 0], hist)
    raw, dropped = maps[1].drain()
    assert dropped == 0
    rec = 16 + CF.OUTLIER_DTYPE.itemsize
    a = np.frombuffer(raw, dtype=np.uint8).reshape(-1, rec)
    idx = a[:, 8:16].copy().view("<u8")[:, 0]
    order = np.argsort(idx, kind="stable")
    assert np.array_equal(idx[order], sel)
    assert np.array_equal(a[order, 16:], recs.view(np.uint8).reshape(len(recs), -1))
    p.destroy()
    for m in maps:
        m.destroy()


def test_batch_64_programs_generated_sizes(ctx):
    """All 64 generated programs over their log-uniform batches (4K-16M events each), one
    persistent launch with the autotuned shape; maps and R0 of every program equal the
    oracle's sequential run over the same events."""
    import paper_2512_12615_gb300 as gx

    progs, sizes = P.batch_programs(), P.batch_sizes()
    items = []
    b = gx.Batch(ctx)
    for p, ((prog, specs, cs), n) in enumerate(zip(progs, sizes)):
        ev = gen.uniform_events(n, seed=0x6758 ^ p)
        gm = [gx.Map.from_spec(ctx, s) for s in specs]
        gp = gx.Program(ctx, prog, gm, cs, deterministic=True, jit=True)
        ret = torch.zeros(n, dtype=torch.int64, device="cuda")
        dev = _dev(ev)
        b.add(gp, dev, n, ret)
        items.append((prog, specs, cs, ev, gm, gp, ret, dev))
    b.plan()
    b.launch()
    torch.cuda.synchronize()

    def oracle_run(k):
        prog, specs, cs, ev = items[k][:4]
        om = O.maps_from_specs(specs)
        r0, _ = O.run(prog, om, ev, cs, want_r0=True)
        return om, r0

    order = sorted(range(len(items)), key=lambda k: -sizes[k])  # longest first
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        futs = {k: ex.submit(oracle_run, k) for k in order}
        for k in range(len(items)):
            om, r0 = futs[k].result()
            _, _, _, _, gm, gp, ret, _ = items[k]
            assert gp.status().status == 0, k
            assert np.array_equal(ret.cpu().numpy(), r0), f"program {k}: R0 differs"
            assert_same(snapshot_gpu(gm), snapshot_oracle(om))
    b.destroy()
    for it in items:
        it[5].destroy()
        for m in it[4]:
            m.destroy()
