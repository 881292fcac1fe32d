"""Pins the oracle's parallel form (`run_parallel`) against its sequential run: the same maps
and ring records on up to 1M events, over 1 to 8 threads, and the same instruction count
where no program path depends on map state.  The merge
descriptions are written here from each program's definition (its docstring or its
listing), not taken from the engine."""
import numpy as np
import pytest

import oracle as O
from tests.asmtext import assemble
from workloads import gen
from workloads import programs as P

U64_ADD = lambda n: [(8 * k, 8, "add") for k in range(n)]  # noqa: E731
# page_heat: heat[region] = {count += w, last_ts = max(ts)} inserted as zeros; tally {warps, bytes} adds
PAGE_HEAT = [{"words": [(0, 8, "add"), (8, 8, "max")], "insert": bytes(16)}, {"words": U64_ADD(2)}]
COUNTING = [{"words": U64_ADD(1)}]
LATENCY = [{"words": U64_ADD(1)}, None]
# the all-operations program of the combining tests, read off its listing
ALLOPS_ARRAY = [(0, 8, "add"), (8, 4, "add"), (16, 8, "or"), (24, 8, "and"), (32, 8, "xor"), (40, 8, "max"),
                (48, 8, "min"), (56, 4, "or"), (60, 4, "xor")]
ALLOPS_HASH = [(0, 8, "add"), (8, 4, "add"), (16, 8, "or"), (32, 8, "xor"), (40, 8, "max"), (60, 4, "xor")]


def sequential(prog, specs, cs, ev, init=None):
    maps = O.maps_from_specs(specs)
    for m, v in zip(maps, init or [None] * len(maps)):
        if v is not None:
            for k in range(m.max_entries):
                m.update(k.to_bytes(4, "little"), v[k * m.value_size:(k + 1) * m.value_size])
    _, count = O.run(prog, maps, ev, cs)
    snaps = []
    for m in maps:
        snaps.append(m.array_values() if m.type == O.MAP_ARRAY else
                     m.hash_items() if m.type == O.MAP_HASH else m.ringbuf_records())
    return snaps, count


def assert_same(specs, a, b):
    for s, x, y in zip(specs, a, b):
        if s["type"] == O.MAP_ARRAY:
            assert np.array_equal(x, y)
        else:
            assert x == y


@pytest.mark.parametrize("threads", [1, 3, 8])
@pytest.mark.parametrize("name", ["counting", "page_heat", "latency"])
def test_parallel_is_sequential(name, threads):
    if name == "counting":
        (prog, specs, cs), ev, merge = P.counting(), gen.uniform_events(200_003, seed=1), COUNTING
    elif name == "page_heat":
        (prog, specs, cs), ev, merge = P.page_heat(), gen.pageheat_events(1 << 20, seed=2), PAGE_HEAT
        ev["size"][::97] = 3
        ev["addr"][7::89] |= np.uint64(1)
    else:
        (prog, specs, cs), ev, merge = P.latency(ring_bytes=1 << 22), gen.latency_pairs(100_001, seed=3), LATENCY
    seq, c_seq = sequential(prog, specs, cs, ev)
    par, c_par = O.run_parallel(prog, specs, ev, cs, merge, threads=threads)
    # page-heat's insert path runs once per part that first meets a key: its instruction
    # count depends on the split; the other programs' paths never look at map state
    assert c_seq == c_par if name != "page_heat" else c_seq <= c_par
    assert_same(specs, seq, par)


def test_every_operation_over_starting_values():
    from tests.test_gpu_shards import ALLOPS, SPECS, allops_events, allops_init

    prog, ev, init = assemble(ALLOPS).prog(), allops_events(50_003, seed=4), allops_init()
    merge = [{"words": ALLOPS_ARRAY}, {"words": ALLOPS_HASH, "insert": bytes(64)}]
    seq, c_seq = sequential(prog, SPECS, 32, ev, init)
    par, c_par = O.run_parallel(prog, SPECS, ev, 32, merge, threads=5, init=init)
    assert c_seq <= c_par  # hash inserts, as in page-heat
    assert_same(SPECS, seq, par)


def test_a_wrong_description_is_caught():
    """Bytes the description leaves out must agree between the parts."""
    prog, specs, cs = P.counting()
    with pytest.raises(ValueError):
        O.run_parallel(prog, specs, gen.uniform_events(10_000, seed=5), cs, [{"words": []}], threads=2)
