"""CPU oracle for the discrete Eikonal system of Eq. 2 (arXiv:1306.4743).

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the
CUDA library: only tests/, ``__graft_entry__.smoke()`` and bench.py's
``cpu_baseline`` / ``--impl reference`` legs may import it.  It shares no
code with ``paper_1306_4743_gb300``; both sides take their inputs from the
seeded generators in ``paper_1306_4743_gb300.workloads``, which hold none of
the method's arithmetic.

Every routine is a thin ctypes call into ``oracle.c`` (plain serial C, FP64).
Arrays follow the grid convention of Sec. 1.1: a grid of nx*ny*nz nodes is a
numpy array of shape (nz, ny, nx), C order, so node (i, j, k) is element
[k, j, i] and linear index i + nx*(j + ny*k).

Parity status: every function here is pinned by tests/test_oracle_*.py
(closed forms, the exact 1D solution, plane waves, brute force on tiny
grids, ordering independence, and the sweep counts of Table 6).
"""
import ctypes
import math

import numpy as np

from .build import build_oracle

_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double


def load_library(path):
    """Open a compiled oracle (liborc.so or a test build of it) and declare
    its signatures."""
    lib = ctypes.CDLL(path)
    lib.orc_local_solve.restype = _D
    lib.orc_local_solve.argtypes = [_D, _D, _D, _D]
    lib.orc_local_solve_textbook.restype = _D
    lib.orc_local_solve_textbook.argtypes = [_D, _D, _D, _D]
    lib.orc_fmm.restype = ctypes.c_int
    lib.orc_fmm.argtypes = [_I64, _I64, _I64, _D, _P, _P, _P, _P, _P]
    lib.orc_value_iteration.restype = ctypes.c_int
    lib.orc_value_iteration.argtypes = [_I64, _I64, _I64, _D, _P, _P, _P,
                                        _P, _I64, _P]
    lib.orc_gauss_seidel_perm.restype = ctypes.c_int
    lib.orc_gauss_seidel_perm.argtypes = [_I64, _I64, _I64, _D, _P, _P,
                                          _P, _P, _P, _I64, _P]
    lib.orc_fsm.restype = ctypes.c_int
    lib.orc_fsm.argtypes = [_I64, _I64, _I64, _D, _P, _P, _P, _P,
                            ctypes.c_int, ctypes.c_int, _D, _D, _I64, _P,
                            _P, _P, _P]
    lib.orc_residual.restype = _D
    lib.orc_residual.argtypes = [_I64, _I64, _I64, _D, _P, _P, _P, _P]
    return lib


_override = None


def _load():
    global _lib
    if _override is not None:
        return _override
    if _lib is None:
        _lib = load_library(build_oracle())
    return _lib


class use_library:
    """Context manager: route every call in this module to another build of
    oracle.c (the mutation tests use it to run the pins against planted
    mistakes)."""

    def __init__(self, lib):
        self.lib = lib

    def __enter__(self):
        global _override
        self.prev = _override
        _override = self.lib
        return self.lib

    def __exit__(self, *exc):
        global _override
        _override = self.prev
        return False


class OracleError(RuntimeError):
    pass


_ERR = {1: "invalid input", 2: "out of memory", 3: "did not converge"}


def _check(rc):
    if rc != 0:
        raise OracleError(_ERR.get(rc, "error %d" % rc))


def _prep(F, mask, q):
    F = np.ascontiguousarray(F, dtype=np.float32)
    if F.ndim != 3:
        raise ValueError("F must have shape (nz, ny, nx)")
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    q = np.ascontiguousarray(q, dtype=np.float64)
    if mask.shape != F.shape or q.shape != F.shape:
        raise ValueError("F, mask and q must share one shape")
    nz, ny, nx = F.shape
    return F, mask, q, nx, ny, nz


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def local_solve(ax, ay, az, s):
    """Root of sum_d max(U - a_d, 0)^2 = s^2 (Eq. 2 at one node)."""
    return _load().orc_local_solve(float(ax), float(ay), float(az), float(s))


def local_solve_textbook(ax, ay, az, s):
    """Same root from the unshifted quadratic (cross-check only)."""
    return _load().orc_local_solve_textbook(float(ax), float(ay), float(az),
                                            float(s))


def fmm(F, mask, q, h, return_stats=False):
    """Serial FP64 Fast Marching Method with a binary heap (Sec. 2)."""
    F, mask, q, nx, ny, nz = _prep(F, mask, q)
    U = np.empty(F.shape, dtype=np.float64)
    nrec = ctypes.c_int64(0)
    _check(_load().orc_fmm(nx, ny, nz, float(h), _ptr(F), _ptr(mask), _ptr(q),
                           _ptr(U), ctypes.byref(nrec)))
    if return_stats:
        return U, {"recomputes": nrec.value}
    return U


def value_iteration(F, mask, q, h, max_iter=100000):
    """Jacobi iteration of U <- min(U, Lambda(U)) from +inf to a bitwise fixed point."""
    F, mask, q, nx, ny, nz = _prep(F, mask, q)
    U = np.empty(F.shape, dtype=np.float64)
    it = ctypes.c_int64(0)
    _check(_load().orc_value_iteration(nx, ny, nz, float(h), _ptr(F),
                                       _ptr(mask), _ptr(q), _ptr(U),
                                       int(max_iter), ctypes.byref(it)))
    return U, it.value


def gauss_seidel(F, mask, q, h, perm, max_pass=100000):
    """Gauss-Seidel passes in the node order `perm` (linear indices) to a fixed point."""
    F, mask, q, nx, ny, nz = _prep(F, mask, q)
    perm = np.ascontiguousarray(perm, dtype=np.int64)
    if perm.shape != (F.size,):
        raise ValueError("perm must list every node once")
    U = np.empty(F.shape, dtype=np.float64)
    it = ctypes.c_int64(0)
    _check(_load().orc_gauss_seidel_perm(nx, ny, nz, float(h), _ptr(F),
                                         _ptr(mask), _ptr(q), _ptr(perm),
                                         _ptr(U), int(max_pass),
                                         ctypes.byref(it)))
    return U, it.value


def fsm(F, mask, q, h, dir_order=(0, 1, 2, 3, 4, 5, 6, 7), inner=0,
        unreached=math.inf, kappa=0.0, max_sweeps=10000,
        allow_unconverged=False):
    """Whole-grid Fast Sweeping (Sec. 2) with per-sweep statistics.

    Returns (U, sweeps, max_change[sweeps], n_changed[sweeps]).  With
    allow_unconverged, stopping at max_sweeps is not an error.
    """
    F, mask, q, nx, ny, nz = _prep(F, mask, q)
    d = np.ascontiguousarray(dir_order, dtype=np.int32)
    U = np.empty(F.shape, dtype=np.float64)
    mc = np.zeros(int(max_sweeps), dtype=np.float64)
    nc = np.zeros(int(max_sweeps), dtype=np.int64)
    sw = ctypes.c_int64(0)
    rc = _load().orc_fsm(nx, ny, nz, float(h), _ptr(F), _ptr(mask), _ptr(q),
                         _ptr(d), len(d), int(inner), float(unreached),
                         float(kappa), int(max_sweeps), _ptr(U),
                         ctypes.byref(sw), _ptr(mc), _ptr(nc))
    if not (allow_unconverged and rc == 3):
        _check(rc)
    s = sw.value
    return U, s, mc[:s].copy(), nc[:s].copy()


def residual(U, F, mask, h):
    """max |U - Lambda(U)| over non-exit nodes, and the count of non-finite U."""
    F = np.ascontiguousarray(F, dtype=np.float32)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    U = np.ascontiguousarray(U, dtype=np.float64)
    nz, ny, nx = F.shape
    bad = ctypes.c_int64(0)
    r = _load().orc_residual(nx, ny, nz, float(h), _ptr(F), _ptr(mask),
                             _ptr(U), ctypes.byref(bad))
    return r, bad.value
