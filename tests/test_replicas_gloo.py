"""The multi-GPU path of bench.py is replicas only (each rank assembles its
own copy; no collective on the data path): the only cross-rank step is the
max over ranks of the timed region and the whole-job rate.  Exercised here
with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank                 # rank 1 is the slowest
    ms_max, value = bench.replica_aggregate(ms, ne=1000, steps=10, world=world, device="cpu")
    out[rank] = (ms_max, value)
    torch.distributed.destroy_process_group()


def test_two_rank_max_and_rate():
    world = 2
    port = _free_port()
    mgr = torch.multiprocessing.get_context("spawn").Manager()
    out = mgr.dict()
    torch.multiprocessing.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        ms_max, value = out[rank]
        assert ms_max == 150.0
        assert value == pytest.approx(world * 1000 * 10 / 0.150)
