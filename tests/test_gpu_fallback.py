"""The replace-mode fallback of the FP32 + FP64-polish mode.

The monotone FP64 polish descends from the FP32 result lifted above the
fixed point (eik_opts.polish_lift, default 2^-11).  If the start were below
the fixed point somewhere, monotone sweeps could not reach it; the residual
check after the polish then queues every cell for replace-mode FP64 sweeps
(u <- Lambda(u), values may rise).  A negative lift starts the polish below
the fixed point everywhere, which forces that path on purpose; its result
must still match the oracle's FMM within the FP32 + polish tolerance, in the
single-grid entry point and in the captured batch graph, where the fallback
is gated on the device.
"""
import numpy as np
import pytest

import oracle
from paper_1306_4743_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BOUND = 1e-9


@pytest.fixture(scope="module")
def eik():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_4743_gb300 import eik as e
    e.load()
    return e


@pytest.mark.parametrize("lift,n", [(-1e-3, 8), (-1e-6, 16), (-2e-2, 8)])
def test_negative_lift_runs_the_fallback_and_matches_oracle(eik, lift, n):
    p = W.oscillatory(67, amp=0.5)
    ref = oracle.fmm(p.F, p.mask, p.q, p.h)
    with eik.Solver(precision="fp32_polish", cell_n=n, polish_lift=lift) as s:
        u, st = s.solve(p.F, p.mask, p.q, p.h, tol=1e-12)
    assert st["fallback_used"] == 1 and st["fallback_visits"] > 0
    assert np.max(np.abs(u - ref)) <= BOUND * np.max(ref)
    assert np.array_equal(u[p.mask == 1], p.q[p.mask == 1])
    assert st["nonfinite"] == 0 and st["residual_max"] <= 1e-11 * st["u_max"]


def test_default_lift_needs_no_fallback(eik):
    p = W.oscillatory(67, amp=0.5)
    with eik.Solver(precision="fp32_polish", cell_n=8) as s:
        _, st = s.solve(p.F, p.mask, p.q, p.h, tol=1e-12)
    assert st["fallback_used"] == 0 and st["fallback_visits"] == 0


def test_fallback_inside_the_captured_batch_graph(eik):
    import torch
    dev = torch.device("cuda", 0)
    probs = W.batch_instances(6)
    bt = [(torch.from_numpy(p.F).to(dev), torch.from_numpy(p.mask).to(dev),
           torch.from_numpy(p.q).to(dev), p.h) for p in probs]
    refs = [oracle.fmm(p.F, p.mask, p.q, p.h) for p in probs]
    with eik.Solver(precision="fp32_polish", polish_lift=-1e-4) as s:
        outs, st = s.solve_batch_device(bt, tol=1e-12)           # plain run, then capture
        for o in outs:
            o.fill_(-1.0)
        outs, st2 = s.solve_batch_device(bt, tol=1e-12, outs=outs)  # graph replay
    for stats in (st, st2):
        assert stats["fallback_used"] == 1 and stats["fallback_visits"] > 0
    for k, (o, ref) in enumerate(zip(outs, refs)):
        assert np.max(np.abs(o.cpu().numpy() - ref)) <= BOUND * np.max(ref), k


def test_lift_outside_its_range_is_rejected(eik):
    with pytest.raises(eik.EikError) as e:
        eik.Solver(precision="fp32_polish", polish_lift=-0.75)
    assert e.value.status == 1
