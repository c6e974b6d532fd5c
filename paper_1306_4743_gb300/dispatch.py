"""Instance sharding across GPUs for batches and serving.

One grid is never split across GPUs (its cells exchange boundary values in
directions known only at run time); independent instances are.  Every rank
computes the same deterministic assignment from the instance sizes alone, so
no collective is needed to agree on it: rank r solves `shard(sizes, r, N)` on
its own GPU and keeps its results.
"""
from __future__ import annotations


def partition(sizes, world: int, budgets=None, bytes_per_node: float = 37.0):
    """Greedy longest-first assignment of instances to `world` ranks.

    sizes: node count of each instance.  Instances are taken in decreasing
    size (ties: lower index first) and each goes to the rank with the least
    assigned nodes (ties: lower rank) among those whose memory budget (bytes,
    per rank, optional) still holds it at `bytes_per_node`.  Returns one
    list of instance indices per rank, each in increasing index order.
    Raises ValueError if an instance fits no rank.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    mem = [0.0] * world
    out = [[] for _ in range(world)]
    order = sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k))
    for k in order:
        need = float(sizes[k]) * bytes_per_node
        best = None
        for r in range(world):
            if budgets is not None and mem[r] + need > budgets[r]:
                continue
            if best is None or load[r] < load[best]:
                best = r
        if best is None:
            raise ValueError("instance %d (%d nodes) fits no rank's budget" % (k, sizes[k]))
        out[best].append(k)
        load[best] += int(sizes[k])
        mem[best] += need
    return [sorted(s) for s in out]


def shard(sizes, rank: int, world: int, budgets=None):
    """The instance indices rank `rank` solves."""
    return partition(sizes, world, budgets)[rank]


def solve_batch_sharded(solver, problems, rank: int, world: int, budgets=None, **kw):
    """Solve this rank's share of `problems` ((F, mask, q, h) tuples) as one
    batch on `solver` (an eik.Solver bound to this rank's GPU).

    Returns ({instance index: u}, stats).  Ranks need not communicate: each
    derives the same split from the instance sizes.
    """
    sizes = []
    for p in problems:
        n = 1
        for e in p[0].shape:
            n *= int(e)
        sizes.append(n)
    mine = shard(sizes, rank, world, budgets)
    if not mine:
        return {}, None
    outs, st = solver.solve_batch([problems[k] for k in mine], **kw)
    return dict(zip(mine, outs)), st
