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


# --- serving across GPUs ------------------------------------------------------
def _serving_sizes(n=120):
    return [e ** 3 for (_, e, _) in W.serving_requests(n=n, rate=1.0, seed=5)]


def test_assign_online_is_greedy_least_loaded_and_deterministic():
    sizes = _serving_sizes()
    for world in (1, 2, 3, 4):
        a = dispatch.assign_online(sizes, world)
        assert a == dispatch.assign_online(sizes, world)
        assert len(a) == len(sizes) and set(a) <= set(range(world))
        loads = [sum(s for s, r in zip(sizes, a) if r == k) for k in range(world)]
        assert max(loads) - min(loads) <= max(sizes)
    # each request went to a rank that was least loaded when it arrived
    load = [0, 0, 0]
    for s, r in zip(sizes, dispatch.assign_online(sizes, 3)):
        assert load[r] == min(load)
        load[r] += s


def test_assign_online_respects_budgets():
    sizes = [100, 10, 100, 10]
    a = dispatch.assign_online(sizes, 2, budgets=[1e9, 50 * 37.0])
    assert a[0] == 0 and a[2] == 0  # the large requests fit rank 0 only
    with pytest.raises(ValueError):
        dispatch.assign_online([1000], 2, budgets=[10.0, 10.0])


class _FakeServer:
    """Stands in for eik.Solver's submit / poll on CPU: a request completes
    after a number of polls that grows with its size, and its 'solution' is
    h, so the caller can tell which request it got."""

    def __init__(self, name):
        self.name = name
        self.req = {}
        self.next = 1
        self.closed = False

    def submit(self, F, mask, q, h, tol=0.0, out=None):
        t = self.next
        self.next += 1
        u = np.full(F.shape, float(h)) if out is None else out
        self.req[t] = [max(1, F.size // 4000), u]
        return t, u

    def poll(self, t):
        r = self.req[t]
        r[0] -= 1
        if r[0] <= 0:
            del self.req[t]
            return True, 0, {"server": self.name}
        return False, 0, {}

    def cancel(self, t):
        return 0 if self.req.pop(t, None) is not None else 9

    def close(self):
        self.closed = True


def _requests(n=40):
    out = []
    for k, (_, e, _) in enumerate(W.serving_requests(n=n, rate=1.0, seed=5)):
        e = max(3, e // 8)  # small stand-ins of the same size mix
        out.append((np.zeros((e, e, e), np.float32), None, None, float(k)))
    return out


def test_sharded_server_balances_outstanding_nodes_and_completes_all():
    reqs = _requests()
    backs = [_FakeServer(i) for i in range(3)]
    srv = dispatch.ShardedServer(backs)
    tickets = {}
    for k, (F, m, q, h) in enumerate(reqs):
        before = list(srv.outstanding)
        t, u = srv.submit(F, m, q, h)
        r = srv.tickets[t][0]
        assert before[r] == min(before)  # least outstanding nodes at submission
        tickets[t] = k
    seen = {}
    while tickets:
        for t in list(tickets):
            done, rc, st = srv.poll(t)
            if done:
                k = tickets.pop(t)
                assert rc == 0 and st["backend"] == st["server"]
                seen[k] = st["backend"]
    assert sorted(seen) == list(range(len(reqs)))
    assert srv.outstanding == [0, 0, 0] and len(set(seen.values())) == 3
    srv.close()
    assert all(b.closed for b in backs)


def test_sharded_server_cancel_and_budget():
    srv = dispatch.ShardedServer([_FakeServer(0), _FakeServer(1)], budgets=[1e12, 8 * 37.0])
    F = np.zeros((4, 4, 4), np.float32)
    t, _ = srv.submit(F, None, None, 1.0)
    assert srv.tickets[t][0] == 0  # 64 nodes do not fit backend 1's budget of 8
    assert srv.cancel(t) == 0 and srv.outstanding == [0, 0]
    with pytest.raises(ValueError):
        dispatch.ShardedServer([_FakeServer(0)], budgets=[1.0]).submit(F, None, None, 1.0)


def _serve_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    reqs = _requests()
    done = dispatch.serve_sharded(_FakeServer(rank), reqs, rank, world)
    # check only: which requests this rank served, and that each got its own
    # answer back (the split itself took no collective)
    mine = torch.full((len(reqs),), -1, dtype=torch.int64)
    for k, (u, rc) in done.items():
        assert rc == 0 and float(u.flat[0]) == float(k)
        mine[k] = rank
    allm = [torch.zeros(len(reqs), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allm, mine)
    dist.destroy_process_group()
    if rank == 0:
        q.put([a.tolist() for a in allm])


def test_two_gloo_ranks_serve_disjoint_covering_shares():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_serve_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    allm = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    reqs = _requests()
    owner = dispatch.assign_online([r[0].size for r in reqs], 2)
    for k in range(len(reqs)):
        served = [r for r in range(2) if allm[r][k] == r]
        assert served == [owner[k]], k
