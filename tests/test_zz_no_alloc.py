"""gx_map_read_noalloc returns the same hash-map snapshot as gx_map_read.

Some callers of this library cannot call cudaMalloc: a control plane whose device-memory
budget is already used up, or a monitoring thread that must not add allocations while
the GPU serves requests.  For them gx_map_read_noalloc compacts a hash map into one
fixed device array instead of a buffer it allocates.  These tests call it through the C
ABI, twice in a row, and compare it with gx_map_read.  They run last (file name) and also
pass alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


SENTINEL = 0xA5


def _noalloc(gx, m, cap):
    buf = np.full(max(cap, 1), SENTINEL, dtype=np.uint8)
    n = ctypes.c_uint64(0)
    rc = gx.lib().gx_map_read_noalloc(m.h, buf.ctypes.data, cap, ctypes.byref(n), None)
    return rc, buf, n.value


def _pairs(raw: bytes, n: int, stride: int):
    return sorted(raw[i * stride:(i + 1) * stride] for i in range(n))


def _fill(m, keys, seed):
    """Writes {key: two random u64} pairs; returns the sorted pairs written."""
    rng = np.random.default_rng(seed)
    vals = rng.integers(0, 1 << 62, size=(len(keys), 2), dtype=np.uint64)
    pairs = [int(k).to_bytes(8, "little") + v.astype("<u8").tobytes() for k, v in zip(keys, vals)]
    m.write(b"".join(pairs))
    return sorted(pairs)


@pytest.fixture(scope="module")
def gx_ctx():
    import paper_2512_12615_gb300 as gx

    return gx, gx.Context(0)


def test_two_calls_match_map_read(gx_ctx):
    gx, ctx = gx_ctx
    big = gx.Map(ctx, gx.MAP_HASH, 8, 16, 1 << 16)
    small = gx.Map(ctx, gx.MAP_HASH, 8, 16, 1024)
    written_big = _fill(big, np.arange(20000, dtype=np.uint64) * 7919 + 3, seed=1)
    written_small = _fill(small, np.arange(300, dtype=np.uint64) + (1 << 40), seed=2)
    # big then small: the second call must not see pairs left over from the first; both
    # snapshots equal the pairs written, and equal gx_map_read's
    for m, written in ((big, written_big), (small, written_small)):
        ref, n_ref = m.read_raw()
        rc, buf, n = _noalloc(gx, m, m.max_entries * 24)
        assert rc == 0 and n == n_ref == len(written)
        assert _pairs(buf[:n * 24].tobytes(), n, 24) == written
        assert _pairs(ref, n_ref, 24) == written
    # two calls in a row on the same map give the same snapshot
    a = _noalloc(gx, big, big.max_entries * 24)
    b = _noalloc(gx, big, big.max_entries * 24)
    assert a[0] == b[0] == 0 and a[2] == b[2] == 20000
    assert _pairs(a[1][:20000 * 24].tobytes(), 20000, 24) == _pairs(b[1][:20000 * 24].tobytes(), 20000, 24)


def test_program_written_map_matches(gx_ctx):
    import torch

    from workloads import gen
    from workloads import programs as P

    gx, ctx = gx_ctx
    prog, specs, cs = P.page_heat(max_entries=1 << 16)
    maps = [gx.Map.from_spec(ctx, s) for s in specs]
    p = gx.Program(ctx, prog, maps, cs, deterministic=True)
    ev = gen.pageheat_events(200_000, seed=5)
    p.run(torch.from_numpy(ev.view(np.uint8).reshape(-1).copy()).cuda(), len(ev))
    torch.cuda.synchronize()
    ref, n_ref = maps[0].read_raw()
    for _ in range(2):
        rc, buf, n = _noalloc(gx, maps[0], maps[0].max_entries * 24)
        assert rc == 0 and n == n_ref > 1000
        assert _pairs(buf[:n * 24].tobytes(), n, 24) == _pairs(ref, n_ref, 24)


def test_limits_are_reported(gx_ctx):
    gx, ctx = gx_ctx
    cap_pairs = ((4 << 20) - 256) // 24  # GX_NOALLOC_SCRATCH_BYTES minus the counter, over the pair size
    m = gx.Map(ctx, gx.MAP_HASH, 8, 16, cap_pairs + 5000)
    _fill(m, np.arange(cap_pairs + 10, dtype=np.uint64), seed=3)
    rc, buf, n = _noalloc(gx, m, m.max_entries * 24)
    assert rc == gx.E2BIG and n == cap_pairs + 10  # more live pairs than the fixed array holds
    assert (buf == SENTINEL).all()  # nothing copied
    small = gx.Map(ctx, gx.MAP_HASH, 8, 16, 64)
    written = _fill(small, np.arange(40, dtype=np.uint64), seed=4)
    rc, buf, n = _noalloc(gx, small, 10 * 24)
    assert rc == gx.E2BIG and n == 40  # caller's buffer too small, though the pairs fit the array
    assert (buf == SENTINEL).all()
    rc, buf, n = _noalloc(gx, small, 40 * 24)  # exactly large enough
    assert rc == 0 and n == 40 and _pairs(buf.tobytes(), 40, 24) == written
    arr = gx.Map(ctx, gx.MAP_ARRAY, 4, 8, 16)
    assert _noalloc(gx, arr, 16 * 8)[0] == gx.EINVAL
