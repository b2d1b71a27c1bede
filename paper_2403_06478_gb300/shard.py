"""Sharding a batch of pairs over several GPUs (one process per GPU).

Every pair is aligned independently, so the alignment has no exchange step:
ranks split the pairs, align their share with the single-GPU path and never
communicate while the kernels run.  The only collectives are host-side: the
gather of the per-pair results and the reduction of the step statistics
(cells summed, times taken at the slowest rank).

The split balances predicted work, not pair counts.  The paper splits its
input into equal parts per GPU and leaves balancing open (Section 5.8); here
each pair's work is estimated with the cell model of Section 4.5 (band cells
= anti-diagonals x band width, about (tlen + qlen)(w + 1)/2) and the pairs are
dealt out longest-processing-time first: each pair, in decreasing order of
work, goes to the least-loaded rank.  That greedy rule keeps the largest load
within 4/3 of the best possible split.
"""
from __future__ import annotations

import heapq
from typing import List, Optional, Sequence

import numpy as np


def predicted_cells(q_len: np.ndarray, t_len: np.ndarray, w: int) -> np.ndarray:
    """Scheduling estimate of each pair's band cells (int64)."""
    q = np.asarray(q_len, dtype=np.int64)
    t = np.asarray(t_len, dtype=np.int64)
    m = np.maximum(q, t)
    we = m if w < 0 else np.minimum(m, w)
    est = (q + t) * (we + 1) // 2
    return np.where((q > 0) & (t > 0), est, 0)


def lpt_partition(work: Sequence[int], n_shards: int) -> List[np.ndarray]:
    """Greedy LPT split of items with the given work into n_shards index sets
    (each sorted ascending).  Ties go to the lowest shard index."""
    if n_shards < 1:
        raise ValueError("n_shards must be >= 1")
    work = np.asarray(work, dtype=np.int64)
    order = np.argsort(-work, kind="stable")
    heap = [(0, s) for s in range(n_shards)]
    parts: List[list] = [[] for _ in range(n_shards)]
    for i in order:
        load, s = heapq.heappop(heap)
        parts[s].append(int(i))
        heapq.heappush(heap, (load + int(work[i]), s))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def shard_indices(q_len, t_len, w: int, rank: int, world: int) -> np.ndarray:
    """The pairs rank `rank` of `world` aligns (every rank computes the same split)."""
    return lpt_partition(predicted_cells(q_len, t_len, w), world)[rank]


def gather_results(local: np.ndarray, local_idx: np.ndarray, n_total: int, group=None) -> np.ndarray:
    """All-gather per-pair result records from every rank into one array in
    batch order.  Works with any torch.distributed backend (gloo, nccl)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts: list = [None] * world
    dist.all_gather_object(parts, (np.asarray(local_idx, dtype=np.int64), local.tobytes()), group=group)
    full = np.zeros(n_total, dtype=local.dtype)
    seen = np.zeros(n_total, dtype=bool)
    for idx, raw in parts:
        rec = np.frombuffer(raw, dtype=local.dtype)
        if rec.shape[0] != idx.shape[0] or seen[idx].any():
            raise RuntimeError("ranks returned overlapping or malformed shards")
        full[idx] = rec
        seen[idx] = True
    if not seen.all():
        raise RuntimeError("some pairs were aligned by no rank")
    return full


def reduce_step_stats(sums: Sequence[float], maxes: Sequence[float], group=None, device=None):
    """Sum `sums` (units processed) and take the max of `maxes` (times) over
    ranks.  Returns two lists of floats."""
    import torch
    import torch.distributed as dist
    s = torch.tensor([float(x) for x in sums], dtype=torch.float64, device=device)
    m = torch.tensor([float(x) for x in maxes], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(m, op=dist.ReduceOp.MAX, group=group)
    return [float(x) for x in s.cpu()], [float(x) for x in m.cpu()]


def align_sharded(ctx, batch, n_shards: int, flags: int = 0, scoring=None) -> np.ndarray:
    """Run the shards of an n_shards-GPU split one after another on this
    context's GPU and reassemble the results in batch order: the single-GPU
    stand-in for the multi-GPU path (same split, same reassembly)."""
    from . import agatha as A
    scoring = scoring if scoring is not None else batch.scoring
    parts = lpt_partition(predicted_cells(batch.q_len, batch.t_len, scoring.w), n_shards)
    out = np.zeros(batch.n_pairs, dtype=A.RESULT_DTYPE)
    for idx in parts:
        if idx.size:
            out[idx] = A.agatha_align_batch(ctx, batch.subset(idx), scoring, flags=flags)
    return out


def load_imbalance(work: Sequence[int], parts: List[np.ndarray]) -> float:
    """Largest shard load over the mean load (1.0 = perfect)."""
    work = np.asarray(work, dtype=np.int64)
    loads = [int(work[p].sum()) for p in parts]
    mean = sum(loads) / max(len(loads), 1)
    return max(loads) / mean if mean else 1.0


def lower_bound(work: Sequence[int], n_shards: int) -> float:
    """A lower bound on the best possible largest load."""
    work = np.asarray(work, dtype=np.int64)
    if work.size == 0:
        return 0.0
    return max(float(work.sum()) / n_shards, float(work.max()))


__all__ = ["predicted_cells", "lpt_partition", "shard_indices", "gather_results",
           "reduce_step_stats", "align_sharded", "load_imbalance", "lower_bound"]

