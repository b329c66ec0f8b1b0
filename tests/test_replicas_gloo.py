"""The N-GPU path of bench.py runs replicas: each rank times its own copy of
the step, the job time is the slowest rank's, and the job's time per atom
counts the atoms of all ranks. Checked with two gloo processes on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
        job_ms = bench.max_over_ranks(ms, dist, "cpu")
        dist.barrier()
        out[rank] = (job_ms, bench.us_per_atom(job_ms, 1000, world))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_atoms():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        job_ms, upa = out[r]
        assert job_ms == 150.0
        assert upa == pytest.approx(150.0 * 1e3 / (1000 * world))


def test_single_process_keeps_its_own_time():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.us_per_atom(12.5, 500, 1) == pytest.approx(25.0)
