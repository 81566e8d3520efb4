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


def test_roofline_takes_the_algorithmic_work_of_each_contraction():
    """The roofline of a contraction counts its algorithmic work only: 2 X n^2 a flops and the
    streamed operand once at 4 bytes plus the output once at 4 bytes for the half transform. The
    split path's own arithmetic peak is the BF16 peak over the nd (nd + 1) / 2 digit products per
    multiply-add. H50 (4 digits) is bound by HBM; H1000 (5 digits) by the tensor cores."""
    import bench
    peaks, _ = bench._peaks()
    bf16 = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    h50 = {"nbf": 150, "naux": 500, "nact": 50}
    r = bench.roofline(1, h50, 1, 0.0455, "GEMM1", nd=4)
    assert r["bound"] == "hbm"
    assert r["algorithmic_bytes"] == 4.0 * 500 * 150 ** 2 + 4.0 * 500 * 150 * 50
    assert abs(r["frac"] - r["algorithmic_bytes"] / 0.0455e-3 / 1e9 / peaks["hbm_gbs"]) < 1e-12
    h1000 = {"nbf": 1000, "naux": 3000, "nact": 1000}
    r = bench.roofline(1, h1000, 1, 140.0, "GEMM1", nd=5)
    assert r["bound"] == "tensor" and r["algorithmic_flops"] == 2.0 * 3000 * 1000 ** 3
    assert abs(r["peak"] - bf16 / 15) < 1e-12
    assert abs(r["frac"] - r["algorithmic_flops"] / 0.140 / 1e12 / (bf16 / 15)) < 1e-12
    assert abs(r["frac_of_bf16_peak_algorithmic"] - r["frac"] / 15) < 1e-12
    # the full transform and the Lagrangian contraction: 2 X n a^2 flops each
    r2 = bench.roofline(1, h1000, 3, 140.0, "GEMM3", nd=5)
    assert r2["algorithmic_flops"] == 2.0 * 3000 * 1000 * 1000 ** 2
    # the whole evaluation: the larger of flops / arithmetic peak and bytes / HBM peak
    e = bench.eval_roofline(1, h1000, 400.0, nd=5)
    flops, nbytes = bench.eval_work(3000, 1000, 1000)
    t = max(flops / (bf16 / 15 * 1e12), nbytes / (peaks["hbm_gbs"] * 1e9))
    assert abs(e["frac"] - t * 1e3 / 400.0) < 1e-12 and e["bound"] == "tensor"
