"""Multi-rank host logic on CPU (gloo, world size 2): the pooled posterior
mean of chains that ran on different ranks, and the max-over-ranks timing
used by bench.py.  No GPU and no collective inside the sampler."""
import os
import socket

import numpy as np
import pytest

from paper_2411_00991_gb300 import dist as D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(rank)
    mean = rng.uniform(1, 5, size=(6, 7))
    count = 10 + 5 * rank
    pooled = D.allreduce_mean(mean, count)
    slow = D.max_over_ranks(1.5 + rank)
    q.put((rank, mean, count, pooled, slow))
    dist.destroy_process_group()


def test_pooled_mean_and_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort(key=lambda x: x[0])
    ref = D.combine_means([o[1] for o in out], [o[2] for o in out])
    for o in out:
        np.testing.assert_allclose(o[3], ref, rtol=1e-15)
        assert o[4] == 2.5


def test_combine_means_weights_by_sweeps():
    a, b = np.full((2, 2), 1.0), np.full((2, 2), 4.0)
    np.testing.assert_array_equal(D.combine_means([a, b], [1, 2]), np.full((2, 2), 3.0))
    with pytest.raises(ValueError):
        D.combine_means([a], [0])
