"""Instance sharding for multi-GPU batches: deterministic, disjoint, covering,
balanced; checked in-process and across two gloo ranks on CPU."""
import os
import socket

import numpy as np
import pytest

from paper_1306_4743_gb300 import dispatch
from paper_1306_4743_gb300 import workloads as W


def test_partition_is_a_balanced_disjoint_cover():
    dims = W.batch_dims(256)
    sizes = [a * b * c for (a, b, c) in dims]
    for world in (1, 2, 3, 4, 8):
        parts = dispatch.partition(sizes, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[k] for k in p) for p in parts]
        # longest-first greedy: every load within one largest instance of the mean
        assert max(loads) - min(loads) <= max(sizes)


def test_partition_respects_budgets():
    sizes = [100, 90, 80, 10, 10]
    parts = dispatch.partition(sizes, 2, budgets=[200 * 37.0, 120 * 37.0])
    assert sum(sizes[k] for k in parts[1]) <= 120
    with pytest.raises(ValueError):
        dispatch.partition([1000], 2, budgets=[10.0, 10.0])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class _RecordingSolver:
    """Stands in for eik.Solver on CPU: returns each instance's index as its
    'solution' so the test sees which rank solved what."""

    def solve_batch(self, batch, **kw):
        return [np.full(b[0].shape, b[3]) for b in batch], {"instances": len(batch)}


def test_solve_batch_sharded_covers_every_instance():
    probs = [(np.zeros(d, np.float32), None, None, float(k))
             for k, d in enumerate(W.batch_dims(20))]
    got = {}
    for r in range(3):
        res, _ = dispatch.solve_batch_sharded(_RecordingSolver(), probs, r, 3)
        assert not set(res) & set(got)
        got.update(res)
    assert sorted(got) == list(range(20))
    assert all(float(got[k].flat[0]) == k for k in got)


def _worker(rank, world, port, sizes, q):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    mine = dispatch.shard(sizes, rank, world)
    # each rank reports what it would solve; no collective decides the split
    n = torch.tensor([len(mine), sum(sizes[k] for k in mine)], dtype=torch.int64)
    got = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(got, n)
    idx = torch.full((len(sizes),), -1, dtype=torch.int64)
    idx[:len(mine)] = torch.tensor(mine, dtype=torch.int64)
    all_idx = [torch.zeros(len(sizes), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_idx, idx)
    dist.destroy_process_group()
    if rank == 0:
        q.put(([g.tolist() for g in got], [[int(v) for v in a if v >= 0] for a in all_idx]))


def test_two_gloo_ranks_agree_on_the_split():
    import torch.multiprocessing as mp
    sizes = [a * b * c for (a, b, c) in W.batch_dims(64)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    counts, shards = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(shards[0] + shards[1]) == list(range(len(sizes)))
    assert shards == dispatch.partition(sizes, 2)
    assert sum(c[1] for c in counts) == sum(sizes)
