"""Multi-process path of bench.py on CPU (gloo, world size 2): every rank solves its
own frequency points (weak scaling, no data-path collective) and the step time is
the maximum over ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pts = [bench.omega_index(rank, world, step, 64) for step in range(5)]
    t = bench.max_over_ranks(dist, 10.0 * (rank + 1))
    bench.barrier(dist)
    q.put((rank, pts, t))
    dist.destroy_process_group()


def test_two_ranks_shard_frequencies_and_take_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, pts0, t0), (r1, pts1, t1) = res
    assert set(pts0).isdisjoint(pts1)                     # no point solved twice
    assert pts0 == [0, 2, 4, 6, 8] and pts1 == [1, 3, 5, 7, 9]
    assert t0 == t1 == 20.0                               # max over ranks


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert [bench.omega_index(0, 1, s, 4) for s in range(6)] == [0, 1, 2, 3, 0, 1]
