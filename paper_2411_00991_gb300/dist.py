"""Multi-process combination of independent chains (one process per GPU).

Chains, images and jobs are independent units of the sampler: ranks share no
data while sweeping.  At the end, the posterior mean of one problem whose
chains ran on several ranks is the sweep-count-weighted double average of the
per-rank means (each rank's mean already pools its own chains), and a timing
is the maximum over ranks.  These helpers do that on the host through
torch.distributed (gloo or nccl); no collective runs inside the sweep.
"""
from __future__ import annotations

import numpy as np


def combine_means(means, counts):
    """Sweep-count-weighted average of per-rank posterior means (double)."""
    counts = np.asarray(counts, dtype=np.float64)
    if counts.sum() <= 0:
        raise ValueError("no averaged sweeps")
    acc = np.zeros_like(np.asarray(means[0], dtype=np.float64))
    for m, n in zip(means, counts):
        acc += np.asarray(m, dtype=np.float64) * n
    return acc / counts.sum()


def allreduce_mean(local_mean: np.ndarray, local_count: int, group=None) -> np.ndarray:
    """All ranks: combine their local means into the pooled mean (double)."""
    import torch
    import torch.distributed as dist
    dev = torch.device("cpu") if dist.get_backend(group) == "gloo" else torch.device("cuda", torch.cuda.current_device())
    w = torch.as_tensor(np.asarray(local_mean, dtype=np.float64) * float(local_count), device=dev)
    n = torch.tensor([float(local_count)], dtype=torch.float64, device=dev)
    dist.all_reduce(w, group=group)
    dist.all_reduce(n, group=group)
    if n.item() <= 0:
        raise ValueError("no averaged sweeps on any rank")
    return (w / n).cpu().numpy()


def max_over_ranks(value: float, group=None) -> float:
    """The maximum of a per-rank scalar (timings are reported as the slowest rank)."""
    import torch
    import torch.distributed as dist
    dev = torch.device("cpu") if dist.get_backend(group) == "gloo" else torch.device("cuda", torch.cuda.current_device())
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
