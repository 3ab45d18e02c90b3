"""Multi-rank host logic on CPU: the cost-balanced batch split and the max-over-ranks
timing reduction, in a world of 2 gloo ranks (127.0.0.1), plus the split's properties
in a single process.  No GPU."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_2608_21227_gb300 import inputs
from paper_2608_21227_gb300.dist import gather_by_index, matrix_cost, max_over_ranks, shard_batch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def check_partition(ms, ns, parts, world):
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(ms)))  # every matrix exactly once
    loads = [sum(matrix_cost(ms[i], ns[i]) for i in p) for p in parts]
    biggest = max((matrix_cost(m, n) for m, n in zip(ms, ns)), default=0.0)
    assert max(loads) - min(loads) <= biggest + 1e-6  # LPT: within one matrix
    assert len(parts) == world


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_batch_properties(world):
    ms, ns = inputs.batch_shapes(1000, seed=3)
    parts = shard_batch(ms, ns, world)
    check_partition(list(ms), list(ns), parts, world)
    assert shard_batch(ms, ns, world) == parts  # deterministic


def test_shard_batch_edges():
    assert shard_batch([], [], 2) == [[], []]
    assert shard_batch([5], [3], 4) == [[0], [], [], []]
    # equal matrices split evenly, lowest ranks first
    assert [len(p) for p in shard_batch([10] * 7, [4] * 7, 3)] == [3, 2, 2]
    with pytest.raises(ValueError):
        shard_batch([1], [1, 2], 2)
    with pytest.raises(ValueError):
        shard_batch([1], [1], 0)


def test_max_over_ranks_single_process():
    assert max_over_ranks(3.5) == 3.5


CHILD = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
from paper_2608_21227_gb300 import inputs
from paper_2608_21227_gb300.dist import max_over_ranks, shard_batch
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:" + os.environ["MASTER_PORT"], rank=rank, world_size=world)
ms, ns = inputs.batch_shapes(500, seed=11)
mine = shard_batch(ms, ns, world)[rank]
t = max_over_ranks(10.0 + rank, dist)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "mine": mine, "max": t}))
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks():
    port = str(free_port())
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=port)
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda o: o["rank"])
    assert [o["max"] for o in outs] == [11.0, 11.0]  # the slowest rank's time on every rank
    ms, ns = inputs.batch_shapes(500, seed=11)
    # the ranks' shares, computed independently, form the same partition as one process's
    assert [o["mine"] for o in outs] == shard_batch(ms, ns, 2)
    check_partition(list(ms), list(ns), [o["mine"] for o in outs], 2)


def test_gather_by_index_single_process():
    assert gather_by_index([2, 0, 1], ["c", "a", "b"], 3) == ["a", "b", "c"]
    with pytest.raises(ValueError):
        gather_by_index([0, 0], ["a", "b"], 2)
    with pytest.raises(ValueError):
        gather_by_index([0], ["a"], 2)


CHILD_BATCH = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch.distributed as dist
import oracle
from paper_2608_21227_gb300 import inputs
from paper_2608_21227_gb300.dist import gather_by_index, shard_batch
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:" + os.environ["MASTER_PORT"], rank=rank, world_size=world)
ms, ns = inputs.batch_shapes(40, seed=21, n_lo=2, n_hi=24)
mine = shard_batch(ms, ns, world)[rank]
# each rank solves only its share (here with the CPU oracle: the host logic is what is tested)
res = [oracle.svdvals(inputs.gaussian(int(ms[i]), int(ns[i]), [21, i])).tolist() for i in mine]
full = gather_by_index(mine, res, len(ms), dist)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "mine": mine, "full": full}))
"""


def test_sharded_batch_end_to_end_two_gloo_ranks():
    # the sharded batched path's host logic: split, per-rank solve of its share, gather back
    port = str(free_port())
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=port)
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD_BATCH, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    import oracle

    ms, ns = inputs.batch_shapes(40, seed=21, n_lo=2, n_hi=24)
    want = [oracle.svdvals(inputs.gaussian(int(ms[i]), int(ns[i]), [21, i])) for i in range(len(ms))]
    assert sorted(outs[0]["mine"] + outs[1]["mine"]) == list(range(len(ms)))
    for o in outs:  # every rank holds the whole batch's results, in batch order
        assert len(o["full"]) == len(ms)
        for got, ref in zip(o["full"], want):
            assert np.array_equal(np.asarray(got), ref)
