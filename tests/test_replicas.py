"""Replica path of bench.py on two CPU ranks (gloo): the job time is the
slowest rank's and the throughput counts every rank's pixels. Images are
independent, so ranks exchange nothing but this one reduction."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = [2.0, 5.0][rank]          # rank 1 is the slow one
        ms, value = bench.replica_throughput(ms_local, 1_000_000, world, torch.device("cpu"))
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
        res = dict(out)
    for rank in (0, 1):
        ms, value = res[rank]
        assert ms == pytest.approx(5.0)
        assert value == pytest.approx(2 * 1_000_000 / 5e-3 / 1e9)


def test_single_process_is_unchanged():
    import bench
    ms, value = bench.replica_throughput(4.0, 8_000_000, 1, None)
    assert ms == 4.0 and value == pytest.approx(8e6 / 4e-3 / 1e9)
