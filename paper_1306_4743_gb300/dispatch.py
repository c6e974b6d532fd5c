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


# ---------------------------------------------------------------------------
# Serving across GPUs.  Requests arrive over time, so the assignment is made
# online, in arrival order, with the rule of `partition`: each request goes
# to the rank with the least nodes assigned so far (ties: lower rank) among
# those whose memory budget can hold the request at all.  The rule depends on
# the request sizes alone, so ranks that see the same request stream agree
# on it without a collective; each rank's own library then admits its
# requests under that rank's HBM budget (eik_submit queues what does not fit
# yet).


def assign_online(sizes, world: int, budgets=None, bytes_per_node: float = 37.0):
    """Rank of each request (node counts `sizes`, in arrival order).
    Raises ValueError if a request exceeds every rank's budget."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    out = []
    for k, n in enumerate(sizes):
        need = float(n) * bytes_per_node
        best = None
        for r in range(world):
            if budgets is not None and need > budgets[r]:
                continue
            if best is None or load[r] < load[best]:
                best = r
        if best is None:
            raise ValueError("request %d (%d nodes) fits no rank's budget" % (k, n))
        out.append(best)
        load[best] += int(n)
    return out


def _nodes(F):
    n = 1
    for e in F.shape:
        n *= int(e)
    return n


def serve_sharded(solver, requests, rank: int, world: int, budgets=None, tol=0.0,
                  poll_sleep=0.0):
    """One rank's part of a served request stream.

    requests: the whole stream as (F, mask, q, h) tuples, the same on every
    rank.  This rank submits the requests that `assign_online` gives it to
    `solver` (an eik.Solver on this rank's GPU, or anything with its
    submit / poll), polls them to completion and returns {request index:
    (u, status)}.  No rank communicates with another.
    """
    import time
    owner = assign_online([_nodes(r[0]) for r in requests], world, budgets)
    pending = {}
    for k, (F, mask, q, h) in enumerate(requests):
        if owner[k] == rank:
            t, u = solver.submit(F, mask, q, h, tol=tol)
            pending[t] = (k, u)
    done = {}
    while pending:
        for t in list(pending):
            ok, rc, _ = solver.poll(t)
            if ok:
                k, u = pending.pop(t)
                done[k] = (u, rc)
        if pending and poll_sleep:
            time.sleep(poll_sleep)
    return done


class ShardedServer:
    """Continuous batching over several GPUs from one host process: one
    backend (an eik.Solver, each on its own device) per GPU.  A submitted
    request goes to the backend with the fewest grid nodes outstanding
    (submitted, not yet completed) among those whose memory budget can hold
    it; each backend batches and admits its requests itself.  Tickets are
    this object's own and map to (backend, backend ticket)."""

    def __init__(self, backends, budgets=None, bytes_per_node: float = 37.0):
        if not backends:
            raise ValueError("at least one backend")
        self.backends = list(backends)
        self.budgets = budgets
        self.bpn = float(bytes_per_node)
        self.outstanding = [0] * len(self.backends)
        self.tickets = {}
        self.next = 1

    def pick(self, nodes):
        need = nodes * self.bpn
        best = None
        for r in range(len(self.backends)):
            if self.budgets is not None and need > self.budgets[r]:
                continue
            if best is None or self.outstanding[r] < self.outstanding[best]:
                best = r
        if best is None:
            raise ValueError("request of %d nodes fits no backend's budget" % nodes)
        return best

    def submit(self, F, mask, q, h, tol=0.0, out=None):
        n = _nodes(F)
        r = self.pick(n)
        bt, u = self.backends[r].submit(F, mask, q, h, tol=tol, out=out)
        t = self.next
        self.next += 1
        self.tickets[t] = (r, bt, n)
        self.outstanding[r] += n
        return t, u

    def poll(self, ticket):
        r, bt, n = self.tickets[ticket]
        done, rc, st = self.backends[r].poll(bt)
        if done:
            del self.tickets[ticket]
            self.outstanding[r] -= n
            st = dict(st)
            st["backend"] = r
        return done, rc, st

    def cancel(self, ticket):
        r, bt, n = self.tickets[ticket]
        rc = self.backends[r].cancel(bt)
        if rc == 0:
            del self.tickets[ticket]
            self.outstanding[r] -= n
        return rc

    def close(self):
        for b in self.backends:
            b.close()
