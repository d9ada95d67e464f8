"""The bench's multi-rank host logic on CPU: two gloo ranks (replicas) report
different step times; every rank must see the slowest one, and the whole-job
throughput counts the bytes of both ranks over that time."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        out[rank] = bench.max_over_ranks(ms, world, device="cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_two_ranks():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1] == 15.0
    # 2 ranks x 1 GB per step x 10 steps over 15 ms
    assert bench.job_throughput(1e9, 10, world, 15.0) == pytest.approx(2 * 1e9 * 10 / 15e-3 / 1e9)
    # one rank: identity, no process group needed
    assert bench.max_over_ranks(7.5, 1) == 7.5
