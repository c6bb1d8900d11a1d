"""The sharded sigma's host logic and collective on CPU ranks (gloo, world size 2).

Sigma is a sum over the terms of H_eff; the library's partition gives every term to
exactly one rank (the same partition on every rank, computed without a device), each
rank sums its own terms and one all-reduce adds the partial sums.  On the CPU the
per-term contributions are seeded stand-in vectors; on a GPU they are the library's
partial sigmas (tests/test_gpu_shard.py).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _work(n=2000, seed=7):
    rng = np.random.default_rng(seed)
    return np.maximum(1, np.exp(rng.normal(16.0, 2.0, n))).astype(np.int64)   # heavy-tailed, like term flops


def _contrib(n_terms, n=4096, seed=8):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_terms, n))


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2501_18263_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _work()
        own = shard.owners(w, world)
        got = [torch.zeros(len(w), dtype=torch.int32) for _ in range(world)]
        dist.all_gather(got, torch.tensor(own, dtype=torch.int32))
        c = _contrib(len(w))
        sig = torch.zeros(c.shape[1], dtype=torch.float64)

        def partial(mine, t):
            t.copy_(torch.from_numpy(c[mine].sum(axis=0)))

        shard.sharded_sum(partial, own, rank, sig)
        out[rank] = (own, [g.numpy() for g in got], sig.numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_two_gloo_ranks_partition_every_term_once_and_sum_to_sigma():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    w = _work()
    c = _contrib(len(w))
    full = c.sum(axis=0)
    own0 = res[0][0]
    for r in range(world):
        own, gathered, sig = res[r]
        assert all(np.array_equal(g, own0) for g in gathered)      # one partition, the same on every rank
        assert np.all((own >= 0) & (own < world))                  # every term to exactly one rank
        assert np.max(np.abs(sig - full)) <= 1e-12 * np.max(np.abs(full))
    load = np.array([w[own0 == r].sum() for r in range(world)])
    assert load.max() - load.min() <= w.max()                       # longest-work-first balance bound


def test_partition_is_deterministic_and_balanced_without_a_device():
    from paper_2501_18263_gb300 import binding as B
    w = _work(500, 3)
    for world in (1, 3, 8):
        a = B.term_partition(w, world)
        b = B.term_partition(w.copy(), world)
        assert np.array_equal(a, b)
        load = np.array([w[a == r].sum() for r in range(world)])
        assert load.sum() == w.sum()
        assert load.max() - load.min() <= w.max()
    # a hand-made case: 5, 4, 3, 3, 1 on two ranks -> {5, 3}, {4, 3, 1}
    assert list(B.term_partition([5, 4, 3, 3, 1], 2)) == [0, 1, 1, 0, 1]
