"""Host-only: the full-size result checks that bench.py applies after its timed steps.

`check_pageheat` and `check_latency` compare device maps and a drained ring with the
closed forms of the policies (tests/closed_forms.py) scaled by the launch count.  Here
they get the oracle's maps after one and two runs over the same batch, and copies with
one value, one key or one ring record changed, which they must refuse.
"""
import numpy as np

import bench
import oracle as O
from workloads import gen
from workloads import programs as P


class Changed:
    """A map whose dump differs from `m` in one place."""

    def __init__(self, m, items=None, array=None):
        self.m, self.items, self.array = m, items, array

    def hash_items(self):
        return self.items if self.items is not None else self.m.hash_items()

    def array_u64(self):
        return self.array if self.array is not None else self.m.array_u64()


def _ring_raw(records):
    """The drained-ring byte stream of [(event index, payload)]: {u32 len; u32 flags; u64 idx}
    then the payload padded to 8 bytes, as the engine's drain returns it."""
    out = bytearray()
    for idx, pay in records:
        out += len(pay).to_bytes(4, "little") + bytes(4) + int(idx).to_bytes(8, "little")
        out += pay + bytes((-len(pay)) % 8)
    return bytes(out)


def test_pageheat_check_accepts_the_oracle_and_refuses_changes():
    prog, specs, cs = P.page_heat(max_entries=1 << 14)
    ev = gen.pageheat_events(30_000, seed=21)
    maps = O.maps_from_specs(specs)
    O.run(prog, maps, ev, cs)
    assert bench.check_pageheat(maps, ev, 1)["ok"]
    assert not bench.check_pageheat(maps, ev, 2)["ok"]  # counts are scaled by the launches
    O.run(prog, maps, ev, cs)
    r = bench.check_pageheat(maps, ev, 2)
    assert r["ok"] and r["keys_differing"] == 0 and r["values_differing"] == 0 and r["tally_ok"]

    items = maps[0].hash_items()
    k = next(iter(items))
    v = bytearray(items[k])
    v[0] ^= 1  # one count
    r = bench.check_pageheat([Changed(maps[0], items={**items, k: bytes(v)}), maps[1]], ev, 2)
    assert not r["ok"] and r["values_differing"] == 1
    fewer = dict(items)
    del fewer[k]  # one key missing
    r = bench.check_pageheat([Changed(maps[0], items=fewer), maps[1]], ev, 2)
    assert not r["ok"] and r["keys_differing"] == 1
    tally = maps[1].array_u64().copy()
    tally[3, 1] += np.uint64(1)  # one tally word
    assert not bench.check_pageheat([maps[0], Changed(maps[1], array=tally)], ev, 2)["tally_ok"]


def test_latency_check_accepts_the_oracle_and_refuses_changes():
    prog, specs, cs = P.latency(ring_bytes=1 << 22)
    ev = gen.latency_pairs(40_000, seed=22)
    maps = O.maps_from_specs(specs)
    O.run(prog, maps, ev, cs)
    recs, dropped = maps[1].ringbuf_records()
    assert dropped == 0 and len(recs) > 100
    raw = _ring_raw(recs)
    r = bench.check_latency(maps, ev, 1, raw, 0)
    assert r["ok"] and r["hist_ok"] and r["ring_ok"] and r["outliers"] == len(recs)
    # records in another order are the same set (they are sorted by pair index)
    assert bench.check_latency(maps, ev, 1, _ring_raw(recs[::-1]), 0)["ok"]
    # a dropped record, a changed payload byte, a reported drop, a changed histogram word
    assert not bench.check_latency(maps, ev, 1, _ring_raw(recs[1:]), 0)["ring_ok"]
    idx, pay = recs[5]
    changed = recs[:5] + [(idx, bytes([pay[0] ^ 1]) + pay[1:])] + recs[6:]
    assert not bench.check_latency(maps, ev, 1, _ring_raw(changed), 0)["ring_ok"]
    assert not bench.check_latency(maps, ev, 1, raw, 1)["ring_ok"]
    hist = maps[0].array_u64().copy()
    hist[np.flatnonzero(hist[:, 0])[0], 0] += np.uint64(1)
    assert not bench.check_latency([Changed(maps[0], array=hist), maps[1]], ev, 1, raw, 0)["hist_ok"]
