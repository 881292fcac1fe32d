"""The N-GPU path's host logic as two gloo ranks on the CPU: weak scaling with no data-path
collective, the slowest rank's time, whole-job throughput, and rank 0 alone reporting."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle as O
        from workloads import gen
        from workloads import programs as P

        # each rank's own batch, its own maps: the same recipe under its own seed
        prog, specs, cs = P.page_heat()
        ev = gen.pageheat_events(4096, seed=bench.rank_seed(rank))
        om = O.maps_from_specs(specs)
        O.run(prog, om, ev, cs)
        heat = sorted(om[0].hash_items().items())
        # the slowest rank sets the job's time
        ms, rate = bench.job_rate(torch, 10.0 + 5.0 * rank, world, 1_000_000)
        out.put((rank, ms, rate, int(ev["addr"][0]), len(heat), sum(v[0] for _, v in heat)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, rate0, a0, k0, c0), (r1, ms1, rate1, a1, k1, c1) = res
    assert (r0, r1) == (0, 1)
    assert ms0 == ms1 == 15.0  # max over ranks
    assert rate0 == rate1 == pytest.approx(2 * 1_000_000 / 0.015 / 1e6)
    assert a0 != a1  # different batches per rank
    assert k0 > 0 and k1 > 0 and c0 > 0 and c1 > 0


def test_single_rank_needs_no_collective():
    import bench

    ms, rate = bench.job_rate(torch, 8.0, 1, 4_000_000)
    assert ms == 8.0 and rate == pytest.approx(500.0)


def test_reference_arm_other_ranks_exit_without_work():
    import bench

    class Args:
        warmup, steps = 3, 1

    assert bench.reference_arm(Args(), 1, 2) == 0


def test_rank_seeds_differ():
    import bench

    assert len({bench.rank_seed(r) for r in range(8)}) == 8 and bench.rank_seed(0) == bench.SEED
