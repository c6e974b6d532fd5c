"""Serving entry points: continuous batching of submitted solves.

Requests of different sizes and speed fields are submitted while others run;
every result matches the oracle, and each result is the same alone and in
the mix (within the FP32 + FP64-polish tolerance).
"""
import time

import numpy as np
import pytest

import oracle
from paper_1306_4743_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def eik():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_4743_gb300 import eik as e
    e.load()
    return e


def _requests():
    reqs = W.serving_requests(n=14, rate=1000.0, seed=5, lo=17, hi=73)
    return [W.serving_problem(edge, seed) for (_, edge, seed) in reqs]


def _drain(solver, tickets, timeout=120.0):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets):
        for t in tickets:
            if t in done:
                continue
            ok, rc, st = solver.poll(t)
            if ok:
                done[t] = (rc, st)
        assert time.time() - t0 < timeout, "serving did not finish"
    return done


def test_mix_matches_oracle_and_alone(eik):
    probs = _requests()
    with eik.Solver(precision="fp32_polish") as s:
        tickets, outs = [], []
        for k, p in enumerate(probs):
            t, u = s.submit(p.F, p.mask, p.q, p.h)
            tickets.append(t)
            outs.append(u)
            if k % 4 == 3:  # poll while requests keep arriving
                s.poll(tickets[0])
        done = _drain(s, tickets)
        for t in tickets:
            assert done[t][0] == 0
        alone = [s.solve(p.F, p.mask, p.q, p.h)[0] for p in probs]
    for p, u, a in zip(probs, outs, alone):
        ref = oracle.fmm(p.F, p.mask, p.q, p.h)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(u - ref)) <= TOL * scale
        assert np.max(np.abs(u - a)) <= TOL * scale
        assert np.array_equal(u[p.mask == 1], p.q[p.mask == 1])


def test_budget_limits_admission_but_everything_finishes(eik):
    probs = _requests()[:6]
    with eik.Solver(precision="fp32_polish", hbm_budget_bytes=48 << 20) as s:
        tickets = [s.submit(p.F, p.mask, p.q, p.h) for p in probs]
        done = _drain(s, [t for t, _ in tickets])
        for (t, u), p in zip(tickets, probs):
            rc = done[t][0]
            assert rc == 0
            ref = oracle.fmm(p.F, p.mask, p.q, p.h)
            assert np.max(np.abs(u - ref)) <= TOL * np.max(ref)
        # a request larger than the whole budget is refused, not hung
        big = W.serving_problem(200, 99)
        t, _ = s.submit(big.F, big.mask, big.q, big.h)
        rc = _drain(s, [t])[t][0]
        assert rc == 3  # EIK_EBUDGET


def test_pinned_buffers_in_place_and_cancel_waits(eik):
    # page-locked inputs are read in place and page-locked outputs written in
    # place; cancelling such a request on the device waits for its batch
    torch = pytest.importorskip("torch")
    probs = _requests()[:6]
    pin = lambda a: torch.from_numpy(a).pin_memory()
    ins = [(pin(p.F), pin(p.mask), pin(p.q)) for p in probs]
    outs = [torch.full(p.F.shape, -1.0, dtype=torch.float64).pin_memory() for p in probs]
    with eik.Solver(precision="fp32_polish") as s:
        tickets = [s.submit(F.numpy(), m.numpy(), q.numpy(), p.h, out=o.numpy())[0]
                   for (F, m, q), o, p in zip(ins, outs, probs)]
        assert s.cancel(tickets[0]) == 0  # likely on the device: returns after its batch
        done = _drain(s, tickets[1:])
        assert all(v[0] == 0 for v in done.values())
    for o, p in zip(outs[1:], probs[1:]):
        u = o.numpy()
        ref = oracle.fmm(p.F, p.mask, p.q, p.h)
        assert np.max(np.abs(u - ref)) <= TOL * np.max(ref)
        assert np.array_equal(u[p.mask == 1], p.q[p.mask == 1])


def test_cancel_waiting_and_running(eik):
    probs = _requests()[:5]
    with eik.Solver(precision="fp32_polish") as s:
        tickets = [s.submit(p.F, p.mask, p.q, p.h)[0] for p in probs]
        assert s.cancel(tickets[-1]) == 0  # likely still waiting
        assert s.cancel(tickets[0]) == 0   # likely on the device
        assert s.cancel(tickets[0]) == 9   # unknown now
        done = _drain(s, tickets[1:-1])
        assert all(v[0] == 0 for v in done.values())
        ok, rc, _ = s.poll(tickets[0])
        assert not ok and rc == 9


def test_sharded_server_over_real_solvers(eik):
    """dispatch.ShardedServer with two library contexts as its backends (both
    on cuda:0 here; on a multi-GPU node each would be one device): requests
    are spread by outstanding nodes, every result matches the oracle, and the
    per-backend counts add up."""
    from paper_1306_4743_gb300 import dispatch
    probs = _requests()
    backs = [eik.Solver(precision="fp32_polish", device=0),
             eik.Solver(precision="fp64", device=0)]
    srv = dispatch.ShardedServer(backs, budgets=[8 << 30, 8 << 30])
    tickets = {}
    for k, p in enumerate(probs):
        t, u = srv.submit(p.F, p.mask, p.q, p.h)
        tickets[t] = (k, u)
    seen = []
    t0 = time.time()
    while tickets:
        for t in list(tickets):
            ok, rc, st = srv.poll(t)
            if ok:
                k, u = tickets.pop(t)
                assert rc == 0, (k, rc)
                p = probs[k]
                ref = oracle.fmm(p.F, p.mask, p.q, p.h)
                bound = TOL if st["backend"] == 0 else 1e-10
                assert np.max(np.abs(u - ref)) <= bound * np.max(ref), k
                seen.append(st["backend"])
        assert time.time() - t0 < 120, "sharded serving did not finish"
    srv.close()
    assert sorted(set(seen)) == [0, 1] and len(seen) == len(probs)
    assert srv.outstanding == [0, 0]
