"""Replica (weak-scaling) host logic of bench.py with two gloo ranks on CPU:
each rank has its own batch and seed, and the job time is the slowest rank's."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 1.0 + rank * 2.5                      # rank 1 is the slow one
        slow = bench.slowest_rank_ms(ms, dist, torch.device("cpu"))
        q.put((rank, slow, bench.rank_seed(rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert [g[1] for g in got] == [3.5, 3.5]
    assert got[0][2] != got[1][2]


def test_single_rank_is_a_no_op():
    assert bench.slowest_rank_ms(2.25, None, "cpu") == 2.25
