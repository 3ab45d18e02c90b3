"""Multi-rank host logic (one process per GPU).

A single matrix does not shard: the panel -> update chain of Algorithm 1 is sequential
step by step, so N GPUs run N independent problems (weak scaling) and nothing on the
data path is exchanged.  Three pieces are shared by the ranks:

- shard_batch: a cost-balanced, deterministic split of a batch of matrices across ranks
  (longest-processing-time-first greedy on the flop count 4mn^2 - 4n^3/3 of each matrix).
  Every rank computes the same partition from the shapes alone, so it needs no
  collective; each rank then makes one nla_gesvd_vals_batched call on its share.
- max_over_ranks: a job's time is its slowest rank's; the benchmark reduces its per-rank
  timings with it (all_reduce MAX over the process group).
- gather_by_index: after the ranks have solved their shares, every rank's (index,
  result) pairs gathered back into batch order -- host objects only (all_gather_object),
  off the timed path; a batch needs no exchange to be solved.
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


def gather_by_index(mine, results, count: int, pg=None):
    """The batch's results in index order from every rank's share.

    `mine` are this rank's batch indices and `results` its results for them (any
    picklable objects, e.g. numpy arrays of singular values).  With no process group
    the share must be the whole batch.  Raises if an index is missing or repeated."""
    pairs = list(zip(mine, results))
    if pg is not None and pg.is_available() and pg.is_initialized() and pg.get_world_size() > 1:
        gathered = [None] * pg.get_world_size()
        pg.all_gather_object(gathered, pairs)
        pairs = [p for part in gathered for p in part]
    out = [None] * count
    seen = [False] * count
    for i, r in pairs:
        if not 0 <= i < count or seen[i]:
            raise ValueError(f"batch index {i} out of range or assigned twice")
        seen[i] = True
        out[i] = r
    if not all(seen):
        raise ValueError("some batch indices were assigned to no rank")
    return out
