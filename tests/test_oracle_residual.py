"""Pins of orc_residual: max |U - Lambda(U)| over the non-exit nodes (Sec. 1.1,
Eq. 2 at each node), and the count of non-finite values.

A residual checker that always returned 0, took a signed difference, counted
exit nodes or skipped a term would pass "zero on FMM solutions" alone, so
these pins feed it non-solutions whose residual is known in closed form:

* the exact 1D solution (U_i = sequential sum of h / F_j from the exit) with
  one interior node raised by delta: Lambda at that node still equals its
  old value, and its downwind neighbour's Lambda rises by delta, so the
  residual is delta (both nodes);
* the same line with its far end node lowered by delta: only that node
  departs from its own Lambda, by -delta, so a signed difference would
  report 0;
* an axis-aligned plane wave (U = i h, F = 1) with one interior node lowered
  by delta: the node and its downwind x neighbour are off by delta, the
  y / z neighbours only by O(delta^2 / h);
* a point source lifted by c away from its exit: Lambda(U + c) = Lambda(U) + c
  wherever the exit is not the smallest neighbour, so the residual is c,
  reached at the six neighbours of the exit;
* an inconsistent exit value (q far above the travel time) is Dirichlet
  data, not an equation: the residual of the FMM solution stays 0;
* non-finite entries are counted, not compared.
"""
import numpy as np

import oracle
from paper_1306_4743_gb300 import workloads as W

ULP = 2.3e-16


def _line(N=40, h=1.0 / 39, i0=5, seed=31):
    """1D grid (N, 1, 1), F uniform in [0.5, 1.5], one exit at i0, and its
    exact solution by sequential sums (the same bits FMM produces)."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.5, 1.5, N).astype(np.float32)
    F = f.reshape(1, 1, N)
    mask = np.zeros(F.shape, np.uint8)
    mask[0, 0, i0] = 1
    q = np.zeros(F.shape)
    s = h / f.astype(np.float64)
    U = np.empty(N)
    U[i0] = 0.0
    for i in range(i0 + 1, N):
        U[i] = U[i - 1] + s[i]
    for i in range(i0 - 1, -1, -1):
        U[i] = U[i + 1] + s[i]
    return F, mask, q, h, U.reshape(F.shape), s


def test_exact_line_has_zero_residual():
    F, mask, q, h, U, _ = _line()
    r, bad = oracle.residual(U, F, mask, h)
    assert (r, bad) == (0.0, 0)


def test_raised_interior_node_gives_delta():
    F, mask, q, h, U, s = _line()
    delta = 1e-3
    assert delta < s.min()
    V = U.copy()
    V[0, 0, 20] += delta
    r, bad = oracle.residual(V, F, mask, h)
    assert bad == 0
    assert abs(r - delta) <= 4 * ULP * U.max()


def test_lowered_end_node_gives_delta():
    # only the last node is off, and by -delta: |.| must be taken
    F, mask, q, h, U, s = _line()
    delta = 2.5e-3
    V = U.copy()
    V[0, 0, -1] -= delta
    r, bad = oracle.residual(V, F, mask, h)
    assert bad == 0
    assert abs(r - delta) <= 4 * ULP * U.max()


def test_lowered_node_of_plane_wave_gives_delta():
    nx, ny, nz, h = 9, 8, 7, 0.125
    F = np.ones((nz, ny, nx), np.float32)
    mask = np.zeros(F.shape, np.uint8)
    mask[:, :, 0] = 1
    q = np.zeros(F.shape)
    U = np.broadcast_to(np.arange(nx) * h, F.shape).copy()
    r0, _ = oracle.residual(U, F, mask, h)
    assert r0 == 0.0
    delta = 1e-4
    V = U.copy()
    V[3, 3, 4] -= delta  # node (i, j, k) = (4, 3, 3)
    r, bad = oracle.residual(V, F, mask, h)
    assert bad == 0
    assert abs(r - delta) <= 8 * ULP
    # the same node on each axis in turn: the y and z neighbours of a lowered
    # node change only to second order, so the maximum is delta whichever
    # axis the wave runs along
    for axis in (1, 2):
        dims = [nx, ny, nz]
        dims[0], dims[axis] = dims[axis], dims[0]
        shape = (dims[2], dims[1], dims[0])
        F2 = np.ones(shape, np.float32)
        m2 = np.zeros(shape, np.uint8)
        coord = np.indices(shape)[2 - axis]
        m2[coord == 0] = 1
        U2 = coord * h
        V2 = U2.astype(np.float64)
        c = [3, 3, 3]
        c[2 - axis] = 4
        V2[tuple(c)] -= delta
        r2, bad2 = oracle.residual(V2, F2, m2, h)
        assert bad2 == 0 and abs(r2 - delta) <= 8 * ULP, axis


def test_lifted_point_source_gives_the_lift():
    p = W.point_source_const(17)
    U = oracle.fmm(p.F, p.mask, p.q, p.h)
    c = 0.25 * p.h
    V = np.where(p.mask == 1, U, U + c)
    r, bad = oracle.residual(V, p.F, p.mask, p.h)
    assert bad == 0
    assert abs(r - c) <= 64 * ULP * U.max()


def test_inconsistent_exit_value_is_not_a_residual():
    F, mask, q, h, _, _ = _line()
    mask[0, 0, 30] = 1
    q[0, 0, 30] = 5.0  # far above the travel time from the first exit
    U = oracle.fmm(F, mask, q, h)
    assert U[0, 0, 30] == 5.0
    r, bad = oracle.residual(U, F, mask, h)
    assert bad == 0 and r == 0.0


def test_nonfinite_entries_are_counted():
    p = W.point_source_const(9)
    U = oracle.fmm(p.F, p.mask, p.q, p.h)
    V = U.copy()
    V[0, 0, 0] = np.inf
    V[8, 8, 8] = np.inf
    V[0, 8, 0] = np.nan
    r, bad = oracle.residual(V, p.F, p.mask, p.h)
    assert bad == 3
    assert np.isfinite(r)
