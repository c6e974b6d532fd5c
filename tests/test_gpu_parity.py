"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: FP64 mode 1e-10 * max(u); FP32 bulk + FP64 polish mode
1e-9 * max(u) -- the accuracy targets of the two precision modes.  Exit
nodes must hold q exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1306_4743_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32_polish": 1e-9}


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def eik():
    _cuda()
    from paper_1306_4743_gb300 import eik as e
    e.load()
    return e


def check_against_oracle(u, p, precision, tol=None):
    ref = oracle.fmm(p.F, p.mask, p.q, p.h)
    umax = float(np.max(np.abs(ref)))
    err = float(np.max(np.abs(u - ref)))
    bound = (tol if tol is not None else TOL[precision]) * max(umax, 1e-300)
    assert np.all(np.isfinite(u))
    assert np.array_equal(u[p.mask == 1], p.q[p.mask == 1])
    assert err <= bound, "max err %.3e > %.3e (umax %.3e)" % (err, bound, umax)
    return err / umax


def random_problem(rng, dims, n_src=3, fmin=0.2, fmax=2.0, qmax=0.3):
    nx, ny, nz = dims
    F = rng.uniform(fmin, fmax, (nz, ny, nx)).astype(np.float32)
    mask = np.zeros(F.shape, np.uint8)
    q = np.zeros(F.shape)
    for t in rng.choice(F.size, n_src, replace=False):
        mask.reshape(-1)[t] = 1
        q.reshape(-1)[t] = rng.uniform(0.0, qmax)
    return W.Problem(F, mask, q, 1.0 / max(max(dims) - 1, 1), "rand%dx%dx%d" % dims)


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
@pytest.mark.parametrize("n", [4, 8, 16])
def test_point_source_small(eik, precision, n):
    p = W.point_source_const(33)
    with eik.Solver(precision=precision, cell_n=n) as s:
        u, st = s.solve(p.F, p.mask, p.q, p.h)
    check_against_oracle(u, p, precision)
    assert st["cell_n_used"] == n and st["cell_visits"] > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
@pytest.mark.parametrize("n", [4, 8, 16])
def test_random_ragged(eik, precision, n):
    rng = np.random.default_rng(100 + n)
    for dims in [(37, 29, 19), (50, 17, 41), (9, 70, 23)]:
        p = random_problem(rng, dims)
        with eik.Solver(precision=precision, cell_n=n) as s:
            u, st = s.solve(p.F, p.mask, p.q, p.h)
        check_against_oracle(u, p, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
def test_exact_1d_and_degenerate_shapes(eik, precision):
    rng = np.random.default_rng(7)
    for dims in [(1, 1, 1), (97, 1, 1), (1, 64, 1), (1, 1, 33), (40, 1, 30), (1, 25, 18)]:
        p = random_problem(rng, dims, n_src=1)
        with eik.Solver(precision=precision, cell_n=8) as s:
            u, _ = s.solve(p.F, p.mask, p.q, p.h)
        check_against_oracle(u, p, precision)
    # exact 1D: sequential sum of h / F from the exit
    N, h = 97, 1.0 / 96
    f = rng.uniform(0.2, 2.0, N).astype(np.float32)
    mask = np.zeros((1, 1, N), np.uint8)
    mask[0, 0, 40] = 1
    with eik.Solver(precision=precision, cell_n=8) as s:
        u, _ = s.solve(f.reshape(1, 1, N), mask, np.zeros((1, 1, N)), h)
    expect = np.zeros(N)
    sv = h / f.astype(np.float64)
    for i in range(41, N):
        expect[i] = expect[i - 1] + sv[i]
    for i in range(39, -1, -1):
        expect[i] = expect[i + 1] + sv[i]
    np.testing.assert_allclose(u.reshape(-1), expect, rtol=1e-14, atol=0)


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
def test_plane_wave(eik, precision):
    nx, ny, nz = 45, 21, 19
    F = np.ones((nz, ny, nx), np.float32)
    mask = np.zeros(F.shape, np.uint8)
    mask[:, :, 0] = 1
    h = 1.0 / 44
    with eik.Solver(precision=precision, cell_n=8) as s:
        u, _ = s.solve(F, mask, np.zeros(F.shape), h)
    expect = np.broadcast_to(np.arange(nx) * h, F.shape)
    np.testing.assert_allclose(u, expect, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
def test_many_sources_and_exit_values(eik, precision):
    rng = np.random.default_rng(11)
    p = random_problem(rng, (48, 40, 36), n_src=40, qmax=2.0)
    with eik.Solver(precision=precision, cell_n=8) as s:
        u, _ = s.solve(p.F, p.mask, p.q, p.h)
    check_against_oracle(u, p, precision)


def test_config1_fp64_65(eik):
    # 65^3 unit cube, F = 1, centre exit, cells of 8^3, kappa = 1e-12
    p = W.point_source_const(65)
    with eik.Solver(precision="fp64", cell_n=8) as s:
        u, st = s.solve(p.F, p.mask, p.q, p.h, tol=1e-12)
    check_against_oracle(u, p, "fp64")
    assert st["residual_max"] <= 1e-11


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
def test_oscillatory_129(eik, precision):
    p = W.oscillatory(129)
    with eik.Solver(precision=precision, cell_n=8) as s:
        u, st = s.solve(p.F, p.mask, p.q, p.h)
    check_against_oracle(u, p, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
@pytest.mark.parametrize("wpc", [4, 6, 8])
def test_worker_shapes_of_16_cubed_cells(eik, precision, wpc):
    # 16^3 cells swept by 4, 6 or 8 warps: the same fixed point
    p = W.oscillatory(97)
    with eik.Solver(precision=precision, cell_n=16, warps_per_cell=wpc) as s:
        u, st = s.solve(p.F, p.mask, p.q, p.h)
    assert st["warps_per_cell_used"] == wpc and st["cell_n_used"] == 16
    check_against_oracle(u, p, precision)


def test_barrier_blocks_129(eik):
    p = W.barrier_blocks(129)
    with eik.Solver(precision="fp32_polish", cell_n=8) as s:
        u, st = s.solve(p.F, p.mask, p.q, p.h)
    check_against_oracle(u, p, "fp32_polish")


def test_invalid_inputs(eik):
    F = np.ones((8, 8, 8), np.float32)
    mask = np.zeros(F.shape, np.uint8)
    q = np.zeros(F.shape)
    with eik.Solver(precision="fp64") as s:
        u, st = s.solve(F, mask, q, 0.1, check=False)
        assert st["status"] == 1  # no exit node
        mask[0, 0, 0] = 1
        F2 = F.copy()
        F2[3, 3, 3] = 0.0
        _, st = s.solve(F2, mask, q, 0.1, check=False)
        assert st["status"] == 1
        F2[3, 3, 3] = np.nan
        _, st = s.solve(F2, mask, q, 0.1, check=False)
        assert st["status"] == 1
        _, st = s.solve(F, mask, q, -0.1, check=False)
        assert st["status"] == 1
        _, st = s.solve(F, mask, q, 0.1, tol=-1.0, check=False)
        assert st["status"] == 1
        # the context is still usable after rejected calls
        u, st = s.solve(F, mask, q, 0.1)
        assert st["status"] == 0 and u[0, 0, 0] == 0.0


# The paper's other workloads (Sec. 6): the rapidly oscillating and the
# strongly curved speeds with the even-grid 8-node exit set, the two
# checkerboards, and the permeable shell maze whose F jumps by 1000x across
# surfaces that cut through cells.
PAPER_WORKLOADS = {
    "ex1_64": lambda: W.paper_example(1, 64),
    "ex2_96": lambda: W.paper_example(2, 96),
    "ex3_80": lambda: W.paper_example(3, 80),
    "checker11_88": lambda: W.checkerboard(88, 11),
    "checker41_84": lambda: W.checkerboard(84, 41),
    "maze_64": lambda: W.shell_maze(64),
}


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
@pytest.mark.parametrize("name", sorted(PAPER_WORKLOADS))
def test_paper_workloads(eik, precision, name):
    p = PAPER_WORKLOADS[name]()
    with eik.Solver(precision=precision) as s:
        u, st = s.solve(p.F, p.mask, p.q, p.h)
    check_against_oracle(u, p, precision)
    assert st["nonfinite"] == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32_polish"])
@pytest.mark.parametrize("name", ["maze_64", "ex2_96", "checker11_88"])
def test_eq4_cell_values(eik, precision, name):
    # The older cell-value heuristic of Sec. 6.8 (Eq. 4, no reset on pop)
    # changes the schedule only: the result is the same fixed point.
    p = PAPER_WORKLOADS[name]()
    with eik.Solver(precision=precision, cell_key=1) as s:
        u, st = s.solve(p.F, p.mask, p.q, p.h)
    check_against_oracle(u, p, precision)
