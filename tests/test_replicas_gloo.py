"""The multi-GPU form of bench.py on the CPU: independent replicas, max over ranks.

The sigma step of one problem is not sharded across GPUs; with N ranks every
rank runs its own replica of the workload and the job's time is the slowest
rank's.  Two gloo ranks check that reduction and the whole-job rate.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
        out[rank] = (ms, bench.job_tflops(2.0e12, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for ms, tf in res.values():
        assert ms == 15.0                                   # the slower rank's time on every rank
        assert abs(tf - 2 * 2.0e12 / 15e-3 / 1e12) < 1e-9    # both replicas' flops in that time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert abs(bench.job_tflops(1e12, 1, 1000.0) - 1.0) < 1e-12
