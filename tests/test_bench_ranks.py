"""The multi-rank host logic of bench.py (replicas, one per GPU) on CPU: two gloo
ranks on 127.0.0.1 agree on the slowest rank's time, and the job's rate is all
ranks' work over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank           # rank 1 is the slower replica
        slowest = bench.max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (slowest, bench.replica_rate(world, 1e12, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slowest, rate = res[0]
    assert slowest == 15.0
    assert rate == pytest.approx(2 * 1e12 / 15e-3)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.replica_rate(1, 3.2e11, 28.0) == pytest.approx(3.2e11 / 28e-3)


def test_preconditioned_loss_roofline_count():
    # n = 1000, d = 2 Gaussian (e = 3d + 1 = 7), p = 3 (w = 4), k = 5 Lanczos
    # steps, 10 CG iterations, rank 20, one second.
    import bench
    rates = {"fp32_ffma2_tflops": 80.0, "mufu_ex2_gops": 10000.0}
    r = bench.precond_lossgrad_roofline(1000, 2, False, 3, 5, 10, 20, 1000.0, rates)
    n, w, e = 1000, 4, 7
    products = n * n * (10 * (2 * w + e) + 5 * (2 * 3 + e) + (4 * w + e + 1))
    nystrom = 2 * 15 * n * 20 ** 2 + n * 20 * 4 * ((10 + 2 * 5 + 1) * 21 + 11 + 20)
    assert r["products_flops"] == products and r["nystrom_flops"] == nystrom
    assert abs(r["achieved_tflops"] - (products + nystrom) / 1e12) < 1e-12
