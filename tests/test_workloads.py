"""The seeded input generators: deterministic, thread-count independent, right shapes."""
import numpy as np

from workloads import gen
from workloads import programs as P


def test_thread_count_invariance():
    for f in (gen.uniform_events, gen.pageheat_events):
        a = f(200_000, seed=5, nthreads=1)
        b = f(200_000, seed=5, nthreads=7)
        assert np.array_equal(a, b)
    a = gen.latency_pairs(100_000, seed=5, nthreads=1)
    assert np.array_equal(a, gen.latency_pairs(100_000, seed=5, nthreads=5))


def test_field_ranges():
    ev = gen.uniform_events(100_000)
    assert ev["addr"].max() < 2**32 and ev["sm_id"].max() <= 147 and ev["warp_id"].max() <= 63
    assert ev["kind"].max() <= 7 and set(np.unique(ev["size"])) == {4, 8, 16, 32}
    assert np.all(np.diff(ev["ts_ns"].astype(np.int64)) >= 1)
    gaps = np.diff(ev["ts_ns"].astype(np.float64))
    assert 950 < gaps.mean() < 1050  # exp(1 us) gaps


def test_pageheat_zipf_head():
    ev = gen.pageheat_events(400_000)
    pages, counts = np.unique(ev["addr"] >> np.uint64(12), return_counts=True)
    # rank-1 probability of Zipf(1.1) over 2^24 items is 1 / H(2^24, 1.1) ~ 0.115
    assert 0.105 < counts.max() / len(ev) < 0.125
    assert ev["addr"].max() < 64 << 30
    assert np.all(ev["addr"] % ev["size"].astype(np.uint64) == 0)


def test_latency_pairs_shape():
    ev = gen.latency_pairs(200_000)
    e, x = ev[0::2], ev[1::2]
    assert np.all(e["kind"] == 0) and np.all(x["kind"] == 1) and np.array_equal(e["addr"], x["addr"])
    lat = (x["ts_ns"] - e["ts_ns"]).astype(np.float64)
    assert 19000 < np.median(lat) < 21000
    t = P.lognormal_quantile_ns(np.log(20000.0), 1.0, 0.99)
    assert abs(t - 204810) < 5
    assert 0.009 < np.mean(lat > t) < 0.011


def test_warp_access_events():
    """Warp-context records: every lane of a warp shares the warp's instruction fields, about
    the requested fraction of warps is coalesced (consecutive size-strided addresses), and
    the output depends on neither the thread count nor anything but the seed."""
    n = 20_000
    ev = gen.warp_access_events(n, seed=9, coalesced=0.75)
    assert np.array_equal(ev, gen.warp_access_events(n, seed=9, coalesced=0.75, nthreads=1))
    assert np.array_equal(ev, gen.warp_access_events(n, seed=9, coalesced=0.75, nthreads=6))
    w = ev.reshape(n, 32)
    for f in ("sm_id", "warp_id", "ts_ns", "kind", "size"):
        assert (w[f] == w[f][:, :1]).all(), f
    raw = ev.view(np.uint8).reshape(-1, 32).reshape(n, 32, 32)
    assert (raw[:, :, gen.WARP_UNIFORM] == raw[:, :1, gen.WARP_UNIFORM]).all()
    step = np.diff(w["addr"].astype(np.int64), axis=1)
    coalesced = (step == w["size"][:, 1:].astype(np.int64)).all(axis=1)
    assert 0.73 < coalesced.mean() < 0.77
    assert np.all(w["addr"] % w["size"].astype(np.uint64) == 0)
    assert np.all(np.diff(w["ts_ns"][:, 0].astype(np.int64)) >= 1)
    assert not gen.warp_access_events(100, seed=9, coalesced=0.0).reshape(100, 32)["addr"].tolist() == \
        gen.warp_access_events(100, seed=9, coalesced=1.0).reshape(100, 32)["addr"].tolist()
    assert len(gen.warp_access_events(7, lanes=5)) == 35
