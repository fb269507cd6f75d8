"""Multi-GPU is replicas only: each rank solves its own copy, the job time is
the slowest rank's, value = ranks x steps / that time.  The host logic of
that path (barrier + max over ranks) runs here on CPU with gloo, 2 ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    elapsed = [2.0, 3.0][rank]  # rank 1 is the slow one
    value, t, w = bench.aggregate_replicas(elapsed, 10, dist, device="cpu")
    out[rank] = (value, t, w)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a threaded test process
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, t, w = res[rank]
        assert w == 2 and t == 3.0
        assert value == pytest.approx(2 * 10 / 3.0)


def test_single_process_aggregation():
    import bench

    value, t, w = bench.aggregate_replicas(4.0, 8, None)
    assert (value, t, w) == (2.0, 4.0, 1)
