"""Entry points and failure paths of the C ABI on the GPU: device-buffer
solves, batches, queue orders, the memory budget, the device wait limit,
and reuse of a context after an error."""
import numpy as np
import pytest

import oracle
from paper_1306_4743_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32_polish": 1e-9}


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def eik(torch):
    from paper_1306_4743_gb300 import eik as e
    e.load()
    return e


def rel_err(u, p):
    ref = oracle.fmm(p.F, p.mask, p.q, p.h)
    return float(np.max(np.abs(u - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("bw", [0.25, 2.0])
def test_queue_orders_and_bucket_widths(eik, precision, order, bw):
    p = W.oscillatory(73, amp=0.5)
    with eik.Solver(precision=precision, cell_n=8, queue_order=order, bucket_width=bw) as s:
        u, st = s.solve(p.F, p.mask, p.q, p.h)
    assert rel_err(u, p) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
def test_device_buffers_match_host_buffers(eik, torch, precision):
    p = W.gaussian_bumps((45, 38, 29), seed=17)
    with eik.Solver(precision=precision, cell_n=8) as s:
        u_h, _ = s.solve(p.F, p.mask, p.q, p.h)
        dev = torch.device("cuda", 0)
        u_d, st = s.solve(torch.from_numpy(p.F).to(dev), torch.from_numpy(p.mask).to(dev),
                          torch.from_numpy(p.q).to(dev), p.h)
    assert rel_err(u_h, p) <= TOL[precision]
    assert rel_err(u_d.cpu().numpy(), p) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
def test_pinned_host_buffers_are_used_in_place(eik, torch, precision):
    # page-locked F and q are read in place and a page-locked u is written in
    # place; the result equals the one from pageable buffers (copied)
    p = W.gaussian_bumps((45, 38, 29), seed=21)
    F, m, q = (torch.from_numpy(a).pin_memory() for a in (p.F, p.mask, p.q))
    out = torch.full(p.F.shape, -1.0, dtype=torch.float64).pin_memory()
    with eik.Solver(precision=precision, cell_n=8) as s:
        s.solve(F.numpy(), m.numpy(), q.numpy(), p.h, out=out.numpy())
        u_pageable, _ = s.solve(p.F, p.mask, p.q, p.h)
    u = out.numpy()
    assert rel_err(u, p) <= TOL[precision]
    assert np.array_equal(u[p.mask == 1], p.q[p.mask == 1])
    assert np.max(np.abs(u - u_pageable)) <= TOL[precision] * np.max(np.abs(u_pageable))


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
def test_batch_matches_single_solves(eik, precision):
    probs = [W.gaussian_bumps(d, 4000 + k) for k, d in
             enumerate([(33, 65, 33), (65, 33, 33), (33, 33, 33), (41, 27, 19), (9, 9, 9)])]
    with eik.Solver(precision=precision, cell_n=8) as s:
        outs, st = s.solve_batch([(p.F, p.mask, p.q, p.h) for p in probs])
    assert st["nodes"] == sum(p.nodes for p in probs)
    for u, p in zip(outs, probs):
        assert rel_err(u, p) <= TOL[precision]
        assert np.array_equal(u[p.mask == 1], p.q[p.mask == 1])


def test_negative_and_mixed_exit_values(eik):
    rng = np.random.default_rng(3)
    F = rng.uniform(0.5, 1.5, (20, 24, 28)).astype(np.float32)
    mask = np.zeros(F.shape, np.uint8)
    q = np.zeros(F.shape)
    for t, v in zip(rng.choice(F.size, 5, replace=False), [-3.0, -2.5, 0.1, 1.0, -2.9]):
        mask.reshape(-1)[t] = 1
        q.reshape(-1)[t] = v
    p = W.Problem(F, mask, q, 0.05)
    for precision in ("fp64", "fp32_polish"):
        with eik.Solver(precision=precision, cell_n=8) as s:
            u, _ = s.solve(p.F, p.mask, p.q, p.h)
        ref = oracle.fmm(p.F, p.mask, p.q, p.h)
        assert np.max(np.abs(u - ref)) <= TOL[precision] * np.max(np.abs(ref))
        assert np.array_equal(u[mask == 1], q[mask == 1])


def test_budget_is_enforced(eik):
    p = W.point_source_const(33)
    with eik.Solver(precision="fp64", hbm_budget_bytes=1 << 16) as s:
        _, st = s.solve(p.F, p.mask, p.q, p.h, check=False)
        assert st["status"] == 3  # EIK_EBUDGET


def test_wait_limit_returns_timeout_and_context_recovers(eik):
    # spin_cap_us = 0: the first idle wait of any worker gives up at once;
    # the kernel ends with EIK_ETIMEOUT instead of waiting
    p = W.point_source_const(41)
    with eik.Solver(precision="fp64", cell_n=8, spin_cap_us=0) as s:
        _, st = s.solve(p.F, p.mask, p.q, p.h, check=False)
        assert st["status"] == 5
    # a fresh context on the same device still solves correctly
    with eik.Solver(precision="fp64", cell_n=8) as s:
        u, st = s.solve(p.F, p.mask, p.q, p.h)
    assert rel_err(u, p) <= 1e-10


def test_context_reuse_across_sizes(eik):
    with eik.Solver(precision="fp32_polish") as s:
        for m in (17, 65, 33, 129, 9):
            p = W.oscillatory(m)
            u, st = s.solve(p.F, p.mask, p.q, p.h)
            assert rel_err(u, p) <= 1e-9
            assert st["cell_n_used"] == (16 if p.nodes >= 2 ** 21 else 8)


def test_stats_are_consistent(eik):
    p = W.oscillatory(65)
    with eik.Solver(precision="fp32_polish", cell_n=8) as s:
        u, st = s.solve(p.F, p.mask, p.q, p.h)
    assert st["nodes"] == p.nodes and st["nonfinite"] == 0
    assert st["cell_visits"] >= (65 // 8 + 1) ** 3 // 2
    assert st["sweeps"] >= st["cell_visits"] and st["polish_sweeps"] >= st["polish_visits"]
    assert st["node_updates"] > 0 and st["polish_node_updates"] > 0
    assert 0 < st["seconds_bulk"] < st["seconds"] and 0 < st["seconds_polish"] < st["seconds"]
    assert st["residual_max"] <= 1e-14 * st["u_max"]
    assert abs(st["u_max"] - u.max()) <= 1e-15 * u.max()
    assert st["kernel_launches"] > 0 and st["grid_ctas"] > 0


def test_autotune_picks_and_applies(eik):
    p = W.oscillatory(49)
    with eik.Solver(precision="fp32_polish") as s:
        n, ctas = s.autotune(p.F, p.mask, p.q, p.h)
        assert n in (4, 8, 16) and ctas > 0
        u, st = s.solve(p.F, p.mask, p.q, p.h)
        assert st["cell_n_used"] == n and st["grid_ctas"] <= ctas
        assert st["warps_per_cell_used"] in ((4, 6, 8) if n == 16 else (1,))
    assert rel_err(u, p) <= 1e-9


def test_default_worker_shapes(eik):
    # 16^3 cells: the FP32 bulk sweeps with 8 warps (one per (j, k) pencil),
    # FP64 sweeps with 6
    p = W.oscillatory(97)
    for precision, wpc in (("fp32_polish", 8), ("fp64", 6)):
        with eik.Solver(precision=precision, cell_n=16) as s:
            u, st = s.solve(p.F, p.mask, p.q, p.h)
        assert st["warps_per_cell_used"] == wpc, precision
        assert rel_err(u, p) <= (1e-9 if precision == "fp32_polish" else 1e-10)


def test_batch_graph_replay_reads_current_inputs(eik, torch):
    dev = torch.device("cuda", 0)
    probs = [W.gaussian_bumps(d, 300 + k) for k, d in enumerate([(33, 33, 65), (41, 29, 23)])]
    bt = [(torch.from_numpy(p.F).to(dev), torch.from_numpy(p.mask).to(dev),
           torch.from_numpy(p.q).to(dev), p.h) for p in probs]
    outs = [torch.empty(p.F.shape, dtype=torch.float64, device=dev) for p in probs]
    with eik.Solver(precision="fp32_polish", cell_n=8) as s:
        for call in range(3):  # plain + capture, then replays of the graph
            outs, st = s.solve_batch_device(bt, outs=outs)
            for u, p in zip(outs, probs):
                assert rel_err(u.cpu().numpy(), p) <= 1e-9, call
        # same buffers, new contents: the replay must solve the new field
        p2 = W.gaussian_bumps((33, 33, 65), 999)
        bt[0][0].copy_(torch.from_numpy(p2.F))
        bt[0][1].copy_(torch.from_numpy(p2.mask))
        bt[0][2].copy_(torch.from_numpy(p2.q))
        outs, st = s.solve_batch_device(bt, outs=outs)
        assert rel_err(outs[0].cpu().numpy(), p2) <= 1e-9
        assert rel_err(outs[1].cpu().numpy(), probs[1]) <= 1e-9


@pytest.mark.parametrize("make", [lambda: W.oscillatory(65), lambda: W.barrier_blocks(65)],
                         ids=["oscillatory65", "barrier65"])
def test_bulk_threshold_from_the_field(eik, make):
    """The FP32 bulk threshold chosen per solve (bulk_kappa_rel = 0) is
    3e-3 r^2 (at most 1) cell edges of front slowness, r = mean(s) mean(1/s)
    over the non-exit nodes, s = h / F; a given factor is used as it is; the
    result meets the FP32 + polish bound either way."""
    p = make()
    s = p.h / p.F[p.mask == 0].astype(np.float64)
    r = float(np.mean(s) * np.mean(1.0 / s))
    s_front = 1.0 / float(np.mean(1.0 / s))
    for rel in (0.0, 0.05):
        with eik.Solver(precision="fp32_polish", bulk_kappa_rel=rel) as sv:
            u, st = sv.solve(p.F, p.mask, p.q, p.h, tol=1e-12)
        factor = rel if rel > 0 else min(3e-3 * r * r, 1.0)
        want = factor * st["cell_n_used"] * s_front
        assert st["bulk_kappa"] == pytest.approx(want, rel=1e-3), (rel, r)
        assert rel_err(u, p) <= TOL["fp32_polish"]
    with eik.Solver(precision="fp64") as sv:
        _, st = sv.solve(p.F, p.mask, p.q, p.h, tol=1e-12)
    assert st["bulk_kappa"] == 0.0
