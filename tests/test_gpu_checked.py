"""The checked interpreter (GX_PROG_CHECKED) on the GPU, through the C ABI.

Every memory access and helper argument is tested against the event's regions before it
is made.  For programs the verifier accepted nothing may fail: the results equal the
oracle's bit for bit, the status is 0 and no access is reported.  (The region tests
themselves are pinned at every edge on the host, tests/test_host_checked.py.)
"""
import json
import os

import numpy as np
import pytest

from tests.asmtext import assemble
from tests.parity import device_events, gpu_maps, run_both
from workloads import gen
from workloads import programs as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    import paper_2512_12615_gb300 as gx

    return gx.Context(0)


def run_checked(ctx, prog, specs, cs, ev, **kw):
    """run_both with a checked program (its status and fault report must stay clear)."""
    run_both(ctx, prog, specs, cs, ev, checked=True, **kw)


@pytest.mark.parametrize("build,events", [(P.counting, lambda: gen.uniform_events(20_011, seed=61)),
                                          (P.page_heat, lambda: gen.pageheat_events(30_007, seed=62)),
                                          (P.latency, lambda: gen.latency_pairs(10_003, seed=63))])
def test_workloads_checked(ctx, build, events):
    prog, specs, cs = build()
    run_checked(ctx, prog, specs, cs, events())


@pytest.mark.parametrize("p", [0, 3, 21, 47, 63])
def test_generated_programs_checked(ctx, p):
    prog, specs, cs = P.batch_programs()[p]
    run_checked(ctx, prog, specs, cs, gen.uniform_events(4099, seed=70 + p))


GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "handworked.json")))["cases"]
ENGINE_CASES = [c for c in GOLDEN if "oracle_only" not in c]


@pytest.mark.parametrize("case", ENGINE_CASES, ids=[c["name"] for c in ENGINE_CASES])
def test_handworked_checked(ctx, case):
    """Rings enlarged to the engine's 4 KiB minimum, as in the unchecked golden test."""
    if case["name"] == "ringbuf_full_drops":
        pytest.skip("needs a 64-byte ring")
    specs = [dict(m) for m in case.get("maps", [])]
    for m in specs:
        if m["type"] == 27:
            m["max_entries"] = max(4096, m["max_entries"])
    ev = np.array(case["events"], dtype=np.uint64)
    run_checked(ctx, assemble(case["asm"]).prog(), specs, 8 * ev.shape[1], ev, det=False)


def test_status_and_refusals(ctx):
    import paper_2512_12615_gb300 as gx

    prog, specs, cs = P.page_heat()
    gm = gpu_maps(ctx, specs)
    p = gx.Program(ctx, prog, gm, cs, deterministic=True, checked=True)
    ev = gen.pageheat_events(5000, seed=64)
    p.run(device_events(ev), len(ev))
    st = p.status()
    assert st.status == 0 and st.fault_pc == 0
    with pytest.raises(gx.GxError) as e:  # checks run in the interpreter only
        gx.Program(ctx, prog, gpu_maps(ctx, specs), cs, jit=True, checked=True)
    assert e.value.status == gx.EINVAL
    b = gx.Batch(ctx)
    with pytest.raises(gx.GxError) as e:  # plain launches only
        b.add(p, device_events(ev), len(ev))
    assert e.value.status == gx.EINVAL
    b.destroy()
