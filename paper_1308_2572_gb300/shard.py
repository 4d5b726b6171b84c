"""Trial-sharded runs over several GPUs, one process per GPU.

Trials are independent (Section III), and the paper's fastest runs split the
trials of the YET between GPUs (Section IV-C). Each rank runs the forward on
one contiguous range of trials; the one exchange is the metrics merge: each
rank reduces its YLT rows to per-layer top-k lists and loss sums (art_topk),
the lists are all-gathered, and the merge selects exactly from their union
(art_merge_topk). This module is host logic and torch.distributed plumbing;
the arithmetic runs in libart.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

from . import art


def trial_range(n_trials: int, world: int, rank: int):
    """Rank's contiguous share [t0, t1) of n_trials trials: the first
    n_trials % world ranks take one trial more."""
    base, extra = divmod(int(n_trials), int(world))
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


def tail_count(p: float, n: int) -> int:
    """k = ceil((1 - p) n), at least 1 and at most n, a (1 - p) n within
    1e-9 n of an integer taken as that integer (the rank art_metrics and
    art_merge_topk use for PML_p and TVaR_p)."""
    if n <= 0:
        return 0
    q = (1.0 - p) * n
    r = float(np.rint(q))
    k = int(r) if abs(q - r) <= 1e-9 * n else int(math.ceil(q))
    return min(n, max(1, k))


def list_length(n_total: int, probs: Sequence[float]) -> int:
    """Top-k list length the merge needs for these probabilities."""
    return max(tail_count(p, n_total) for p in probs)


def gather_lists(top, sums, group=None):
    """All-gather every rank's top-k lists [L][k] and loss sums [L] (torch
    tensors on the rank's device: CUDA with NCCL, CPU with gloo); returns
    host arrays [S][L][k] and [S][L] in rank order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    tops = [torch.empty_like(top) for _ in range(world)]
    sms = [torch.empty_like(sums) for _ in range(world)]
    dist.all_gather(tops, top.contiguous(), group=group)
    dist.all_gather(sms, sums.contiguous(), group=group)
    return (np.ascontiguousarray(torch.stack(tops).cpu().numpy()),
            np.ascontiguousarray(torch.stack(sms).cpu().numpy()))


def merge(top_all, sums_all, n_total: int, probs: Sequence[float]):
    """Mean [L], PML and TVaR [L][n_p] of the whole YLT from the gathered
    lists (art_merge_topk, on the host)."""
    S, L, k = top_all.shape
    n_p = len(probs)
    mean = np.empty(L)
    pml = np.empty((L, n_p))
    tvar = np.empty((L, n_p))
    art.art_merge_topk(np.ascontiguousarray(top_all, dtype=np.float64),
                       np.ascontiguousarray(sums_all, dtype=np.float64), S, L, k, n_total, probs, mean, pml, tvar)
    return mean, pml, tvar


def sharded_metrics(ylt_shard, n_total: int, probs: Sequence[float], group=None, stream=None):
    """The metrics of a YLT whose trials are split between the ranks: this
    rank's rows ylt_shard (CUDA float64 [L][T_rank]) reduced on its GPU, the
    lists gathered, merged on the host. Every rank gets the same results."""
    import torch
    L, T = ylt_shard.shape
    k = list_length(n_total, probs)
    top = torch.empty((L, k), dtype=torch.float64, device=ylt_shard.device)
    sums = torch.empty(L, dtype=torch.float64, device=ylt_shard.device)
    art.art_topk(ylt_shard, T, L, k, top, sums, stream)
    top_all, sums_all = gather_lists(top, sums, group)
    return merge(top_all, sums_all, n_total, probs)
