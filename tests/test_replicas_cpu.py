"""Multi-process path of bench.py on the CPU: two gloo ranks (127.0.0.1).
Replicas are timed by the slowest rank and credited with the work of all
ranks: reduce_over_ranks gives every rank the maximum of the times and the
sum of the proposal counts; without a process group it returns its input."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch
    import bench
    torch.distributed.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                                         rank=rank, world_size=world)
    try:
        ms = [5.0, 7.5][rank]
        props = [1000, 1200][rank]
        q.put((rank, bench.reduce_over_ranks(torch, ms, "max"),
               bench.reduce_over_ranks(torch, props, "sum")))
    finally:
        torch.distributed.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 7.5, 2200.0), (1, 7.5, 2200.0)]


def test_reduce_over_ranks_without_group():
    import torch
    import bench
    assert bench.reduce_over_ranks(torch, 3.25, "max") == 3.25
    assert bench.reduce_over_ranks(torch, 17, "sum") == 17
