"""Seeded synthetic inputs for the Eikonal solver: speed fields F, exit masks
and exit values q on uniform grids.

This module holds input data only, none of the solver's arithmetic: it is
the one piece that both the CUDA library's callers and the CPU oracle use,
so that both sides solve identical problems.  Every random draw takes an
explicit seed (numpy PCG64).

Grid convention (Sec. 1.1): node (i, j, k) sits at x = (i h, j h, k h); a
grid of nx*ny*nz nodes is a numpy array of shape (nz, ny, nx), C order.

Workloads
---------
* ``paper_example(e, m)``: the paper's three benchmark speeds on an m^3 grid
  of the unit cube (h = 1/(m-1)), with the exit set taken as the 8 nodes
  nearest the centre when m is even, or the centre node when m is odd
  (Sec. 6, "Benchmark problems").
* ``point_source_const(m)``: unit cube, m^3 nodes, F = 1, exit at the centre
  node (odd m) -- the 65^3 FP64 workload.
* ``oscillatory(m, freq)``: F = 1 + 0.5 sin(freq x) sin(freq y) sin(freq z),
  exit at the centre node -- the 257^3 workload uses freq = 4 pi.
* ``barrier_blocks(m, blocks, p_slow, f_slow, n_src, field_seed, src_seed)``:
  the unit cube cut into blocks^3 boxes, each slow (F = f_slow) with
  probability p_slow, else F = 1; n_src exit nodes drawn from nodes in fast
  boxes -- the 513^3 workload (16 blocks, p = 0.3, F = 0.01, 8 exits).
* ``gaussian_bumps(dims, seed)``: F = clip(1 + sum of 8 Gaussian bumps,
  0.2, 2) on a box whose longest axis spans [0, 1], one random exit node --
  the instances of the batch and serving workloads.
* ``batch_instances(count, base_seed)``: per-axis edges drawn i.i.d. from
  {33, 65, 129}, instance k seeded base_seed + k.
* ``serving_requests(n, rate, seed)``: Poisson arrival times and cubic edges
  log-uniform in [33, 385].
* ``checkerboard(m, K)`` and ``shell_maze(m)``: the piecewise-constant speeds
  of Sec. 6.6-6.7.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Problem:
    """One Eikonal instance: speed F (nz, ny, nx) float32, exit mask uint8,
    exit values q float64 (read only where mask != 0), grid step h."""
    F: np.ndarray
    mask: np.ndarray
    q: np.ndarray
    h: float
    name: str = ""

    @property
    def dims(self):
        nz, ny, nx = self.F.shape
        return (nx, ny, nz)

    @property
    def nodes(self) -> int:
        return int(self.F.size)


def _axes(m, h):
    return np.arange(m, dtype=np.float64) * h


def _grid_coords(nx, ny, nz, h):
    x = _axes(nx, h)[None, None, :]
    y = _axes(ny, h)[None, :, None]
    z = _axes(nz, h)[:, None, None]
    return x, y, z


def _exits(shape, nodes, values=None):
    mask = np.zeros(shape, dtype=np.uint8)
    q = np.zeros(shape, dtype=np.float64)
    for t, (i, j, k) in enumerate(nodes):
        mask[k, j, i] = 1
        q[k, j, i] = 0.0 if values is None else values[t]
    return mask, q


def centre_exits(m):
    """Exit nodes nearest the cube centre: the centre node (odd m) or the
    8 surrounding nodes (even m), as in Sec. 6."""
    if m % 2:
        c = [m // 2]
    else:
        c = [m // 2 - 1, m // 2]
    return [(i, j, k) for k in c for j in c for i in c]


def point_source_const(m: int = 65) -> Problem:
    h = 1.0 / (m - 1)
    F = np.ones((m, m, m), dtype=np.float32)
    mask, q = _exits(F.shape, centre_exits(m))
    return Problem(F, mask, q, h, "const_%d" % m)


def oscillatory(m: int = 257, freq: float = 4.0 * math.pi,
                amp: float = 0.5) -> Problem:
    h = 1.0 / (m - 1)
    x, y, z = _grid_coords(m, m, m, h)
    F = (1.0 + amp * np.sin(freq * x) * np.sin(freq * y) * np.sin(freq * z))
    F = F.astype(np.float32)
    mask, q = _exits(F.shape, centre_exits(m))
    return Problem(F, mask, q, h, "osc_%d" % m)


def paper_example(e: int, m: int) -> Problem:
    """Sec. 6 examples: 1) F = 1; 2) F = 1 + .5 sin(20 pi x) sin(20 pi y)
    sin(20 pi z); 3) F = 1 + .99 sin(2 pi x) sin(2 pi y) sin(2 pi z)."""
    if e == 1:
        p = point_source_const(m)
    elif e == 2:
        p = oscillatory(m, 20.0 * math.pi, 0.5)
    elif e == 3:
        p = oscillatory(m, 2.0 * math.pi, 0.99)
    else:
        raise ValueError("example is 1, 2 or 3")
    p.name = "ex%d_%d" % (e, m)
    return p


def barrier_blocks(m: int = 513, blocks: int = 16, p_slow: float = 0.3,
                   f_slow: float = 0.01, n_src: int = 8, field_seed: int = 3,
                   src_seed: int = 33) -> Problem:
    """Unit cube in blocks^3 boxes; box b of node i is min(floor(blocks*x), blocks-1)."""
    h = 1.0 / (m - 1)
    rng = np.random.default_rng(field_seed)
    slow = rng.random((blocks, blocks, blocks)) < p_slow  # [bz, by, bx]
    b = np.minimum(np.floor(blocks * _axes(m, h)).astype(np.int64), blocks - 1)
    box_slow = slow[b[:, None, None], b[None, :, None], b[None, None, :]]
    F = np.where(box_slow, np.float32(f_slow), np.float32(1.0)).astype(np.float32)
    fast_nodes = np.flatnonzero(~box_slow.ravel())
    srng = np.random.default_rng(src_seed)
    pick = srng.choice(fast_nodes, size=n_src, replace=False)
    nodes = [(int(t % m), int((t // m) % m), int(t // (m * m))) for t in pick]
    mask, q = _exits(F.shape, nodes)
    return Problem(F, mask, q, h, "barrier_%d" % m)


def gaussian_bumps(dims, seed: int, n_bumps: int = 8) -> Problem:
    """F = clip(1 + sum_k a_k exp(-|x - c_k|^2 / (2 sigma_k^2)), 0.2, 2) with
    c_k uniform in the box, a_k ~ U[-1, 1], sigma_k ~ U[0.05, 0.2]; one exit
    node uniform over the grid with q = 0.  h = 1/(max edge - 1)."""
    nx, ny, nz = (int(d) for d in dims)
    h = 1.0 / (max(nx, ny, nz) - 1)
    rng = np.random.default_rng(seed)
    ext = np.array([(nx - 1) * h, (ny - 1) * h, (nz - 1) * h])
    cen = rng.random((n_bumps, 3)) * ext
    amp = rng.uniform(-1.0, 1.0, n_bumps)
    sig = rng.uniform(0.05, 0.2, n_bumps)
    x, y, z = _grid_coords(nx, ny, nz, h)
    F = np.ones((nz, ny, nx), dtype=np.float64)
    for t in range(n_bumps):
        # exp(-|x - c|^2 / 2 sigma^2) is a product of three 1D factors
        c = -1.0 / (2.0 * sig[t] ** 2)
        gx = np.exp(c * (x - cen[t, 0]) ** 2)
        gy = np.exp(c * (y - cen[t, 1]) ** 2)
        gz = amp[t] * np.exp(c * (z - cen[t, 2]) ** 2)
        F += (gz * gy) * gx
    F = np.clip(F, 0.2, 2.0).astype(np.float32)
    src = int(rng.integers(0, nx * ny * nz))
    node = (src % nx, (src // nx) % ny, src // (nx * ny))
    mask, q = _exits(F.shape, [node])
    return Problem(F, mask, q, h, "bumps_%dx%dx%d_s%d" % (nx, ny, nz, seed))


def batch_dims(count: int = 256, base_seed: int = 4000,
               edges=(33, 65, 129)):
    """Per-instance (nx, ny, nz), each edge drawn i.i.d. from `edges`."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(base_seed + k)
        out.append(tuple(int(e) for e in rng.choice(np.asarray(edges), 3)))
    return out


def batch_instances(count: int = 256, base_seed: int = 4000,
                    edges=(33, 65, 129)):
    """The batch workload: instance k has dims from batch_dims and a
    speed field from gaussian_bumps seeded base_seed + k."""
    return [gaussian_bumps(d, base_seed + k)
            for k, d in enumerate(batch_dims(count, base_seed, edges))]


def serving_requests(n: int = 500, rate: float = 100.0, seed: int = 5,
                     base_seed: int = 5000, lo: int = 33, hi: int = 385):
    """Poisson arrivals: returns a list of (arrival_time_s, edge, seed) with
    exponential inter-arrival gaps of mean 1/rate and cubic edge
    round(exp(U[ln lo, ln hi]))."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n)
    t = np.cumsum(gaps)
    edges = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), n)))
    return [(float(t[k]), int(edges[k]), base_seed + k) for k in range(n)]


def serving_problem(edge: int, seed: int) -> Problem:
    return gaussian_bumps((edge, edge, edge), seed)


def checkerboard(m: int, K: int) -> Problem:
    """Sec. 6.6: the unit cube in K^3 checkers of edge 1/K, F = 2 on one
    colour and 1 on the other, exit set at the centre."""
    h = 1.0 / (m - 1)
    b = np.minimum(np.floor(K * _axes(m, h)).astype(np.int64), K - 1)
    par = (b[:, None, None] + b[None, :, None] + b[None, None, :]) % 2
    F = np.where(par == 0, np.float32(2.0), np.float32(1.0)).astype(np.float32)
    mask, q = _exits(F.shape, centre_exits(m))
    return Problem(F, mask, q, h, "checker%d_%d" % (K, m))


def shell_maze(m: int, t: float = 1.0 / 12.0, w: float = 0.1,
               f_barrier: float = 0.001) -> Problem:
    """Sec. 6.7: domain [-1, 1]^3, exit at the origin, four concentric
    spherical barriers of thickness t (F = f_barrier inside) with openings
    x^2 + y^2 < w on alternating sides."""
    h = 2.0 / (m - 1)
    c = -1.0 + np.arange(m, dtype=np.float64) * h
    x = c[None, None, :]
    y = c[None, :, None]
    z = c[:, None, None]
    r = np.sqrt(x * x + y * y + z * z)
    hole = (x * x + y * y) < w
    barrier = np.zeros((m, m, m), dtype=bool)
    for r0, below in ((0.3, True), (0.5, False), (0.7, True), (0.9, False)):
        shell = (r > r0) & (r < r0 + t)
        opening = hole & ((z < 0) if below else (z > 0))
        barrier |= shell & ~opening
    F = np.where(barrier, np.float32(f_barrier), np.float32(1.0)).astype(np.float32)
    mask, q = _exits(F.shape, centre_exits(m))
    return Problem(F, mask, q, h, "maze_%d" % m)
