"""The replica path of bench.py on two CPU ranks (gloo): the whole-job value
is all ranks' units over the slowest rank's time; no other collective."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_s = 2.0 if rank == 0 else 3.0  # rank 1 is the slow one
    t, value = bench.replica_value(local_s, 1000.0, world, "cpu")
    out[rank] = (t, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_reduction():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, value = res[rank]
        assert t == 3.0
        assert abs(value - 2 * 1000.0 / 3.0) < 1e-9


def test_single_rank_is_local():
    import bench
    t, value = bench.replica_value(4.0, 100.0, 1)
    assert t == 4.0 and value == 25.0
