"""Host logic of the multi-rank benchmark on CPU: two gloo ranks act as replicas; the job time is
the slowest rank's and the throughput sums every rank's evaluations."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [100.0, 250.0][rank]
    value, t_max = bench.aggregate(ms_local, 40, world, dist, device="cpu")
    out[rank] = (value, t_max)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_sum_work():
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        value, t_max = out[rank]
        assert t_max == 250.0
        assert value == pytest.approx(2 * 40 / 0.25)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.aggregate(200.0, 10, 1) == (50.0, 200.0)
