"""The benchmark's multi-GPU path on CPU: two gloo ranks run the host logic
that bench.py runs under torchrun (replicas, weak scaling, no data-path
collective): each rank's seeds, the max-over-ranks timing and the whole-job
value."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.rank_seeds(rank, 16)
        own = 10.0 + 5.0 * rank                     # this rank's time (ms)
        ms = bench.max_over_ranks(own, "cpu")
        val = bench.whole_job_mpoints(world, 16, 2048 * 2048, ms * 1e-3)
        q.put((rank, seeds, ms, val))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (r0, s0, ms0, v0), (r1, s1, ms1, v1) = out
    assert (r0, r1) == (0, 1)
    assert s0 == list(range(0, 16)) and s1 == list(range(16, 32))     # disjoint fields per rank
    assert ms0 == ms1 == 15.0                                        # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 16 * 2048 * 2048 / 15e-3 / 1e6)


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.rank_seeds(0, 3) == [0, 1, 2]
