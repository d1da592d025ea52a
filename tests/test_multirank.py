"""The multi-rank path of the benchmark on CPU: two gloo ranks shard the
events (disjoint blocks, no data exchange) and reduce the slowest rank's
time; the whole-job rate counts every rank's events."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench
    from synth import events as E
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n_ev = 2
    first = bench.shard_first_event(rank, n_ev)
    b = E.make_batch("pu50-ttbar-like", n_events=n_ev, first=first)
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    q.put((rank, first, int(b["x"].size), float(b["x"][:8].sum()), slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_events_and_reduce_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), q), nprocs=world, join=True, start_method="spawn")
    got = sorted(q.get() for _ in range(world))
    assert [g[1] for g in got] == [0, 2]                       # disjoint consecutive event blocks
    assert got[0][2] != got[1][2] or got[0][3] != got[1][3]    # different events
    assert all(g[4] == 15.0 for g in got)                      # every rank sees the slowest time


def test_whole_job_rate_counts_every_rank():
    import bench
    assert np.isclose(bench.whole_job_rate(64, 4, 10.0), 64 * 4 / 0.010)
    assert bench.max_over_ranks(3.0, 1) == 3.0
