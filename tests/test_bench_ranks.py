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


def test_roofline_counts_the_digits_of_the_operands():
    """GEMM1's algorithmic work on the split path: 2 nd bytes per element of B plus the
    double-float T, and nd (nd + 1) / 2 BF16 products. H50 (4 digits) is bound by HBM; H200
    (5 digits) by the tensor cores, against the sustained BF16 peak."""
    import bench
    h50 = {"nbf": 150, "naux": 500, "nact": 50}
    r = bench.roofline(2, h50, 0.0455, "GEMM1", nd=4)
    assert r["bound"] == "hbm" and r["algorithmic_bytes"] == 8.0 * 500 * 150 ** 2 + 8.0 * 500 * 150 * 50
    peaks, _ = bench._peaks()
    assert abs(r["frac"] - r["algorithmic_bytes"] / 0.0455e-3 / 1e9 / peaks["hbm_gbs"]) < 1e-12
    h200 = {"nbf": 600, "naux": 2000, "nact": 200}
    r = bench.roofline(2, h200, 9.0, "GEMM1", nd=5)
    assert r["bound"] == "tensor" and r["algorithmic_flops"] == 15 * 2.0 * 2000 * 600 ** 2 * 200
    assert r["algorithmic_bytes"] == 10.0 * 2000 * 600 ** 2 + 8.0 * 2000 * 600 * 200
    assert r["peak"] == peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
