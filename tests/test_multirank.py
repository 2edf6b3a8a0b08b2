"""The N > 1 path of bench.py: N independent replicas (one workload per rank, no data
exchange), timed by the slowest rank.  Two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    value, t = bench.replica_throughput(units_local=16 * 10, t_local=times[rank], dist=dist, device="cpu")
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    world, port = 2, _free_port()
    times = [2.0, 3.0]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, t = res[r]
        assert t == 3.0                                  # the slowest rank's time
        assert value == pytest.approx(world * 160 / 3.0)  # all ranks' units over it


def test_replica_throughput_single_process():
    import bench
    value, t = bench.replica_throughput(160, 2.0)
    assert (value, t) == (80.0, 2.0)
