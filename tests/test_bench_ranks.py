"""bench.py's multi-rank host logic (replicas, max-over-ranks timing) on two
gloo ranks on the CPU: every rank sees the slowest rank's time and the
whole-job rate counts every rank's work."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    w, r, local = bench.dist_init()
    dist.init_process_group("gloo", rank=r, world_size=w)
    bench.barrier(w)
    t = bench.reduce_max(100.0 + 7.0 * r, w)  # rank r "took" 100 + 7r ms
    q.put((r, local, t, bench.job_rate(w, 5, 2, t)))
    bench.barrier(w)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_timing_two_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = 100.0 + 7.0 * (world - 1)
    for r, (rank, local, t, rate) in enumerate(got):
        assert rank == r and local == r
        assert t == slowest
        assert rate == pytest.approx(world * 5 * 2 / (slowest / 1e3))


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.job_rate(1, 10, 1, 100.0) == pytest.approx(100.0)
