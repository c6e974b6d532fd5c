"""The allocation-free entry point eik_solve_device_noalloc, called through
the C ABI, gives the same values as the ordinary FP64 device entry point
(eik_solve_device) and as the CPU oracle's FMM, within the FP64 tolerance of
the parity tests, on consecutive calls that share its fixed scratch array.

Callers that cannot allocate device memory during a solve (a program whose
own caching allocator holds the device memory, a latency-critical loop, a
plug-in limited to the memory it is handed) use this entry point; the test
itself allocates freely, the entry point does not.  This file is collected
last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1306_4743_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_4743_gb300 import eik
    return torch, eik, eik.load()


def _dev(torch, p):
    d = torch.device("cuda", 0)
    return (torch.from_numpy(p.F).to(d), torch.from_numpy(p.mask).to(d),
            torch.from_numpy(p.q).to(d))


def _noalloc(torch, eik, lib, p, F, m, q):
    u = torch.full(p.F.shape, -1.0, dtype=torch.float64, device=F.device)
    nz, ny, nx = p.F.shape
    dims = (ctypes.c_int64 * 3)(nx, ny, nz)
    st = eik.Stats()
    stream = torch.cuda.current_stream(F.device).cuda_stream
    rc = lib.eik_solve_device_noalloc(dims, float(p.h), F.data_ptr(), m.data_ptr(), q.data_ptr(),
                                      0.0, u.data_ptr(), ctypes.c_void_p(stream),
                                      ctypes.byref(st))
    return rc, u, st


def test_noalloc_matches_device_entry_point_on_consecutive_calls(env):
    torch, eik, lib = env
    problems = [W.oscillatory(57, amp=0.5), W.gaussian_bumps((41, 30, 23), 9),
                W.oscillatory(57, amp=0.5)]
    with eik.Solver(precision="fp64", cell_n=8) as solver:
        for p in problems:
            F, m, q = _dev(torch, p)
            ref, _ = solver.solve(F, m, q, p.h)
            rc, u, st = _noalloc(torch, eik, lib, p, F, m, q)
            assert rc == 0, eik.STATUS_NAMES.get(rc, rc)
            torch.cuda.synchronize()
            un, rn = u.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(un))
            assert np.max(np.abs(un - rn)) <= TOL_FP64 * np.max(np.abs(rn))
            fmm = oracle.fmm(p.F, p.mask, p.q, p.h)
            assert np.max(np.abs(un - fmm)) <= TOL_FP64 * np.max(fmm)
            assert np.array_equal(un[p.mask == 1], p.q[p.mask == 1])
            assert st.nodes == p.nodes and st.cell_visits > 0
            assert st.kernel_launches == 8


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    torch, eik, lib = env
    d = torch.device("cuda", 0)
    tiny_f = torch.ones(1, device=d, dtype=torch.float32)
    tiny_m = torch.ones(1, device=d, dtype=torch.uint8)
    tiny_q = torch.zeros(1, device=d, dtype=torch.float64)
    tiny_u = torch.zeros(1, device=d, dtype=torch.float64)
    dims = (ctypes.c_int64 * 3)(400, 400, 400)  # rejected before any device access
    rc = lib.eik_solve_device_noalloc(dims, 0.01, tiny_f.data_ptr(), tiny_m.data_ptr(),
                                      tiny_q.data_ptr(), 0.0, tiny_u.data_ptr(), None, None)
    assert rc == 3  # EIK_EBUDGET
