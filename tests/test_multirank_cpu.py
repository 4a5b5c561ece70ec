"""The multi-GPU path runs independent replicas (no collective in the data
path); the only communication is the timing reduction.  Check it with two
gloo ranks on the CPU: every rank sees the max step time, and the whole-job
value counts the points of both ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = [10.0, 14.0][rank]
    ms, value, ws = bench.combine_ranks(ms_local, pts_per_rank=1000, steps=5, dist=dist, device="cpu")
    results[rank] = (ms, value, ws)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_total_points():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.start_processes(_worker, args=(world, port, results), nprocs=world, start_method="spawn", join=True)
        res = dict(results)
    for rank in range(world):
        ms, value, ws = res[rank]
        assert ws == 2
        assert ms == pytest.approx(14.0)
        assert value == pytest.approx(2 * 1000 * 5 / 0.014)


def test_single_process_is_identity():
    import bench

    ms, value, ws = bench.combine_ranks(8.0, pts_per_rank=10, steps=4)
    assert (ms, ws) == (8.0, 1) and value == pytest.approx(10 * 4 / 0.008)
