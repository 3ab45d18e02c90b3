"""Multi-rank host logic (one process per GPU).

A single matrix does not shard: the panel -> update chain of Algorithm 1 is sequential
step by step, so N GPUs run N independent problems (weak scaling) and nothing on the
data path is exchanged.  Two pieces are shared by the ranks:

- shard_batch: a cost-balanced, deterministic split of a batch of matrices across ranks
  (longest-processing-time-first greedy on the flop count 4mn^2 - 4n^3/3 of each matrix).
  Every rank computes the same partition from the shapes alone, so it needs no
  collective; each rank then makes one nla_gesvd_vals_batched call on its share.
- max_over_ranks: a job's time is its slowest rank's; the benchmark reduces its per-rank
  timings with it (all_reduce MAX over the process group).
"""
from __future__ import annotations

import heapq


def matrix_cost(m: int, n: int) -> float:
    """Flops of the singular values of an m x n matrix (4 M N^2 - 4 N^3 / 3, M >= N)."""
    big, small = max(int(m), int(n)), min(int(m), int(n))
    return 4.0 * big * small * small - 4.0 * small ** 3 / 3.0


def shard_batch(ms, ns, world: int):
    """Indices of the batch assigned to each rank: a list of `world` ascending index lists.

    Matrices are taken largest first (ties by index) and each goes to the rank with the
    least work so far (ties by rank), so every rank's load is within one matrix of the
    others'.  Deterministic: every rank computes the same split."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if len(ms) != len(ns):
        raise ValueError("ms and ns differ in length")
    order = sorted(range(len(ms)), key=lambda i: (-matrix_cost(ms[i], ns[i]), i))
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + matrix_cost(ms[i], ns[i]), r))
    return [sorted(p) for p in parts]


def max_over_ranks(value: float, pg=None, device=None) -> float:
    """The largest `value` over the ranks of the default process group (`pg` is the
    torch.distributed module, or None for a single process)."""
    if pg is None or not pg.is_available() or not pg.is_initialized() or pg.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())
