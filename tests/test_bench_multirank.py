"""The multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2) on 127.0.0.1.

Each rank solves its own Gram (weak scaling, no data-path collective); the only exchange is the
max-over-ranks reduction of the timed milliseconds, after which rank 0 reports the whole-job
throughput.  Ranks draw different synthetic paths of the same shape.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 100.0 + 25.0 * rank  # rank 1 is the slow one
        total = bench.max_over_ranks(my_ms, dist, torch.device("cpu"))
        X, Y = bench.workload(rank, n=4, points=9)
        dist.barrier()
        out.put((rank, total, bench.job_throughput(1000, world, 10, total), X.sum(), X.shape))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_slowest_time_and_draw_their_own_paths():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, t0, v0, s0, sh0), (_, t1, v1, s1, sh1) = res
    assert t0 == t1 == 125.0
    assert v0 == v1 == 1000 * 2 * 10 / 0.125
    assert sh0 == sh1 == (4, 9, bench.D)
    assert not np.isclose(s0, s1)  # independent data per rank


def test_single_rank_keeps_its_own_time():
    assert bench.max_over_ranks(42.0, None, None) == 42.0
    assert bench.job_throughput(10, 1, 2, 1000.0) == 20.0
