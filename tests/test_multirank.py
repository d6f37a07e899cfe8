"""The multi-rank (torchrun) path of bench.py on CPU: world size 2 over gloo.

Each rank processes its own batch (weak scaling, no collective in the data
path); the only collective is the max of the per-rank times."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    mx = bench.reduce_max_ms(times[rank], dist)
    value = bench.whole_job_rate(4096, w, 10, mx)
    out[rank] = (mx, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_weak_scaling():
    world = 2
    times = [12.5, 20.0]
    out = mp.Manager().dict()
    mp.start_processes(_rank, args=(world, _free_port(), times, out), nprocs=world, start_method="spawn")
    for r in range(world):
        mx, value = out[r]
        assert mx == max(times)
        assert value == pytest.approx(world * 4096 * 10 / (max(times) / 1e3))


def test_single_rank_is_identity():
    assert bench.reduce_max_ms(7.0, None) == 7.0
    assert bench.whole_job_rate(4096, 1, 10, 1000.0) == pytest.approx(40960.0)
