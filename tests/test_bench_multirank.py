"""The bench's multi-rank host logic on CPU: two gloo ranks, the job's time is
the slowest rank's and the value counts every rank's units (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    import bench
    # rank 1 is slower: 3 steps of 20 ms against rank 0's 3 of 10 ms
    step_ms = [10.0, 10.0, 10.0] if rank == 0 else [20.0, 20.0, 20.0]
    value, total_s = bench.job_throughput(step_ms, world, 4096 * 500)
    out[rank] = (value, total_s)
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_takes_the_slowest_rank_and_counts_all_units():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        value, total_s = out[r]
        assert total_s == pytest.approx(0.060)                     # max over ranks
        assert value == pytest.approx(2 * 4096 * 500 * 3 / 0.060)   # whole-job units / job time


def test_single_rank_needs_no_process_group():
    import bench
    value, total_s = bench.job_throughput([5.0, 5.0], 1, 100)
    assert total_s == pytest.approx(0.010) and value == pytest.approx(2 * 100 / 0.010)
