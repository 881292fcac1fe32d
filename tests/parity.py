"""Runs one program on the oracle and on the engine over the same events and compares.

Bit-exact comparison (the results are integers): R0 of every event, array maps word for
word, hash maps as {key: value} sets, ring-buffer records sorted by event index (records
of one event keep their emission order).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np

import oracle as O
import paper_2512_12615_gb300 as gx


def device_events(ev: np.ndarray):
    import torch

    raw = np.ascontiguousarray(ev).view(np.uint8).reshape(-1)
    t = torch.from_numpy(raw.copy()).cuda()
    assert t.data_ptr() % 16 == 0
    return t


def gpu_maps(ctx: gx.Context, specs: Sequence[dict]) -> List[gx.Map]:
    return [gx.Map.from_spec(ctx, s) for s in specs]


def snapshot_gpu(maps: Sequence[gx.Map]):
    out = []
    for m in maps:
        if m.type == gx.MAP_ARRAY:
            out.append(("array", m.array_values().copy()))
        elif m.type == gx.MAP_HASH:
            out.append(("hash", m.hash_items()))
        else:
            raw, dropped = m.drain()
            recs = gx.parse_records(raw)
            recs = sorted(enumerate(recs), key=lambda t: (t[1][0], t[0]))
            out.append(("ring", [r for _, r in recs], dropped))
    return out


def snapshot_oracle(maps: Sequence[O.Map]):
    out = []
    for m in maps:
        if m.type == O.MAP_ARRAY:
            out.append(("array", m.array_values().copy()))
        elif m.type == O.MAP_HASH:
            out.append(("hash", m.hash_items()))
        else:
            recs, dropped = m.ringbuf_records()
            out.append(("ring", recs, dropped))
    return out


def assert_same(gpu_snap, ora_snap) -> None:
    assert len(gpu_snap) == len(ora_snap)
    for i, (g, o) in enumerate(zip(gpu_snap, ora_snap)):
        assert g[0] == o[0]
        if g[0] == "array":
            if not np.array_equal(g[1], o[1]):
                bad = np.nonzero((g[1] != o[1]).any(axis=1))[0]
                raise AssertionError(f"map {i}: array differs at {len(bad)} entries, first {bad[:8].tolist()}")
        elif g[0] == "hash":
            if g[1] != o[1]:
                gk, ok_ = set(g[1]), set(o[1])
                diff = [k for k in gk & ok_ if g[1][k] != o[1][k]]
                raise AssertionError(f"map {i}: hash differs: only gpu {len(gk - ok_)}, only oracle {len(ok_ - gk)}, "
                                     f"value diffs {len(diff)}")
        else:
            assert g[2] == o[2], f"map {i}: drops {g[2]} vs {o[2]}"
            assert len(g[1]) == len(o[1]), f"map {i}: {len(g[1])} records vs {len(o[1])}"
            assert g[1] == o[1], f"map {i}: ring records differ"


def run_both(ctx: gx.Context, prog: np.ndarray, specs: Sequence[dict], ctx_size: int, events: np.ndarray, *,
             det: bool = True, launch: Optional[Tuple[int, ...]] = None, idx_base: int = 0, check_r0: bool = True,
             jit: bool = False, init: Optional[Sequence[Optional[bytes]]] = None, checked: bool = False):
    """Returns (gpu snapshot, oracle snapshot, r0 gpu, r0 oracle) after asserting equality.

    init: per map, None or the initial values of an array map (max_entries * value_size bytes)."""
    import torch

    n = np.ascontiguousarray(events).view(np.uint8).size // ctx_size
    om = O.maps_from_specs(specs)
    for i, blob in enumerate(init or []):
        if blob is not None:
            vs = specs[i]["value_size"]
            for k in range(specs[i]["max_entries"]):
                assert om[i].update(k.to_bytes(4, "little"), blob[k * vs:(k + 1) * vs]) == 0
    r0_o, _ = O.run(prog, om, events, ctx_size, want_r0=True, event_idx_base=idx_base)
    gm = gpu_maps(ctx, specs)
    for i, blob in enumerate(init or []):
        if blob is not None:
            gm[i].write(blob)
    p = gx.Program(ctx, prog, gm, ctx_size, deterministic=det, jit=jit, checked=checked)
    dev = device_events(events)
    ret = torch.zeros(max(n, 1), dtype=torch.int64, device="cuda")
    p.run(dev, n, ret_out=ret, idx_base=idx_base, launch=launch)
    torch.cuda.synchronize()
    st = p.status()
    assert st.status == 0 and st.fault_pc == 0, (st.status, st.fault_pc)
    r0_g = ret[:n].cpu().numpy()
    gs, os_ = snapshot_gpu(gm), snapshot_oracle(om)
    if check_r0:
        if not np.array_equal(r0_g, r0_o):
            bad = np.nonzero(r0_g != r0_o)[0]
            raise AssertionError(f"R0 differs at {len(bad)} events, first {bad[:8].tolist()}: "
                                 f"gpu {r0_g[bad[:4]].tolist()} oracle {r0_o[bad[:4]].tolist()}")
    assert_same(gs, os_)
    p.destroy()
    for m in gm:
        m.destroy()
    return gs, os_, r0_g, r0_o
