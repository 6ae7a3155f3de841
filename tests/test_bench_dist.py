"""The multi-rank bookkeeping of bench.py (replicas only: a barrier and a max
over ranks of the timed region) on world_size 2 with gloo on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    d = bench.dist_init("gloo")
    bench.barrier(d)
    t_ms = 100.0 + 50.0 * rank  # rank 1 is the slowest
    t_max = bench.reduce_max(d, t_ms, torch.device("cpu"))
    v = bench.throughput(world, 10, t_max)
    q.put((rank, t_max, v, bench.dist_env()))
    d.destroy_process_group()


def test_two_rank_max_timing_and_aggregate_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, v, env in out:
        assert t_max == 150.0
        # all ranks' channels over the slowest rank's time: 2 x 8 x 10 / 0.15 s
        assert v == pytest.approx(2 * 8 * 10 / 0.150)
        assert env == (rank, 2, rank)


def test_throughput_counts_the_plans_channels():
    """pairs/s = ranks x channels x steps / seconds, with the channel count
    of the plan timed (64 for the mixed-precision workload), not the
    headline's 8."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.throughput(1, 10, 1000.0) == bench.NBATCH * 10
    assert bench.throughput(2, 5, 500.0, nbatch=64) == 2 * 64 * 5 / 0.5
