"""The multi-replica timing of bench.py on two gloo ranks on the CPU: every rank gets the
slowest rank's time, and the whole-job rate counts the iterations of every rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = 1.0 + 0.5 * rank  # rank 1 is the slow one
    t = bench.max_over_ranks(mine, torch.device("cpu"))
    out[rank] = (t, bench.whole_job_rate(10, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0] == out[1] == (1.5, pytest.approx(20 / 1.5))


def test_single_process_returns_local_time():
    import torch
    import bench
    assert bench.max_over_ranks(2.5, torch.device("cpu")) == 2.5
    assert bench.whole_job_rate(30, 1, 1.5) == pytest.approx(20.0)
