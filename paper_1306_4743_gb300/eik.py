"""Python binding of libeik.so (C ABI in include/eik.h).

Argument marshalling only: every step of a solve runs in the CUDA library.
There is no CPU fallback -- if libeik.so cannot be built or loaded, every
call raises.

Arrays follow the grid convention of the paper (Sec. 1.1): a grid of
nx*ny*nz nodes is an array of shape (nz, ny, nx), C order, so node (i,j,k)
is element [k, j, i].

    from paper_1306_4743_gb300 import eik
    with eik.Solver(precision="fp32_polish") as s:
        u, stats = s.solve(F, mask, q, h, tol=0.0)      # numpy in, numpy out
        u_dev, stats = s.solve(F_t, mask_t, q_t, h)     # torch CUDA tensors in/out
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libeik.so")

EIK_OK = 0
STATUS_NAMES = {0: "EIK_OK", 1: "EIK_EINVAL", 2: "EIK_ENOMEM", 3: "EIK_EBUDGET",
                4: "EIK_ECUDA", 5: "EIK_ETIMEOUT", 6: "EIK_ENOCONV",
                7: "EIK_ECANCELLED", 8: "EIK_EQUEUE", 9: "EIK_ENOTFOUND"}
PRECISIONS = {"fp64": 0, "fp32_polish": 1}

# Every C entry point declared in include/eik.h.
EXPORTED = ("eik_opts_default", "eik_create", "eik_destroy", "eik_strerror",
            "eik_solve", "eik_solve_device", "eik_solve_batch",
            "eik_solve_batch_device", "eik_submit", "eik_poll", "eik_cancel",
            "eik_solve_device_noalloc", "eik_autotune", "eik_struct_sizes",
            "eik_selftest_local_solve", "eik_dfsm_solve_device")


class Opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("precision", ctypes.c_int),
                ("cell_n", ctypes.c_int), ("max_ctas", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t),
                ("spin_cap_us", ctypes.c_uint64),
                ("bucket_width", ctypes.c_double),
                ("max_sweeps_per_visit", ctypes.c_int),
                ("queue_order", ctypes.c_int),
                ("bulk_kappa_rel", ctypes.c_double),
                ("use_graphs", ctypes.c_int), ("cell_key", ctypes.c_int),
                ("warps_per_cell", ctypes.c_int), ("serve_batch_nodes", ctypes.c_uint64),
                ("polish_lift", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double),
                ("cell_visits", ctypes.c_uint64), ("sweeps", ctypes.c_uint64),
                ("node_updates", ctypes.c_uint64),
                ("polish_visits", ctypes.c_uint64),
                ("polish_sweeps", ctypes.c_uint64),
                ("polish_node_updates", ctypes.c_uint64),
                ("queue_pushes", ctypes.c_uint64),
                ("nonfinite", ctypes.c_uint64), ("nodes", ctypes.c_uint64),
                ("cell_n_used", ctypes.c_int), ("precision_used", ctypes.c_int),
                ("residual_max", ctypes.c_double), ("u_max", ctypes.c_double),
                ("seconds_bulk", ctypes.c_double),
                ("seconds_polish", ctypes.c_double),
                ("kernel_launches", ctypes.c_uint64),
                ("grid_ctas", ctypes.c_int), ("fallback_used", ctypes.c_int),
                ("busy_seconds_bulk", ctypes.c_double),
                ("busy_seconds_polish", ctypes.c_double),
                ("fallback_visits", ctypes.c_uint64),
                ("phase_seconds", (ctypes.c_double * 4) * 2),
                ("revisits", ctypes.c_uint64 * 2),
                ("revisit_sweeps", ctypes.c_uint64 * 2),
                ("revisit_updates", ctypes.c_uint64 * 2),
                ("max_visit_sweeps", ctypes.c_uint64 * 3),
                ("seconds_stage", ctypes.c_double * 3),
                ("warps_per_cell_used", ctypes.c_int), ("reserved_stats", ctypes.c_int),
                ("bulk_kappa", ctypes.c_double)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if name == "phase_seconds":
                v = [[v[i][j] for j in range(4)] for i in range(2)]
            elif name in ("revisits", "max_visit_sweeps", "revisit_sweeps", "revisit_updates"):
                v = [int(x) for x in v]
            elif name == "seconds_stage":
                v = [float(x) for x in v]
            d[name] = v
        return d


class EikError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        name = STATUS_NAMES.get(status, str(status))
        super().__init__("%s%s (%s)" % (where + ": " if where else "", name,
                                        _strerror(status)))


_lib = None


def _strerror(status):
    try:
        return load().eik_strerror(status).decode()
    except Exception:  # the library itself may be what failed
        return "status %d" % status


def load(path: str | None = None):
    """Load libeik.so (building it in-tree with nvcc if it is missing or
    stale).  Raises if the library cannot be produced: there is no fallback."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    if path is None:
        from . import _build
        path = _build.build_eik()
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.eik_opts_default.argtypes = [ctypes.POINTER(Opts)]
    lib.eik_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Opts)]
    lib.eik_destroy.argtypes = [P]
    lib.eik_strerror.argtypes = [I]
    lib.eik_strerror.restype = ctypes.c_char_p
    lib.eik_solve.argtypes = [P, P, D, P, P, P, D, P, ctypes.POINTER(Stats)]
    lib.eik_solve_device.argtypes = [P, P, D, P, P, P, D, P, P, ctypes.POINTER(Stats)]
    lib.eik_solve_batch.argtypes = [P, I, P, P, P, P, P, D, P, ctypes.POINTER(Stats)]
    lib.eik_solve_batch_device.argtypes = [P, I, P, P, P, P, P, D, P, P,
                                           ctypes.POINTER(Stats)]
    lib.eik_submit.argtypes = [P, P, D, P, P, P, D, P, ctypes.POINTER(ctypes.c_uint64)]
    lib.eik_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(I), ctypes.POINTER(Stats)]
    lib.eik_cancel.argtypes = [P, ctypes.c_uint64]
    lib.eik_solve_device_noalloc.argtypes = [P, D, P, P, P, D, P, P, ctypes.POINTER(Stats)]
    lib.eik_autotune.argtypes = [P, P, D, P, P, P, D, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.eik_selftest_local_solve.argtypes = [I, I64, ctypes.c_uint64, ctypes.POINTER(D),
                                             ctypes.POINTER(D)]
    lib.eik_dfsm_solve_device.argtypes = [P, D, P, P, P, D, I64, P, P,
                                          ctypes.POINTER(I64), P, P,
                                          ctypes.POINTER(Stats)]
    lib.eik_struct_sizes.argtypes = [ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t)]
    for name in EXPORTED:
        if name != "eik_strerror":
            getattr(lib, name).restype = I
    so, ss = ctypes.c_size_t(), ctypes.c_size_t()
    lib.eik_struct_sizes(ctypes.byref(so), ctypes.byref(ss))
    if (so.value, ss.value) != (ctypes.sizeof(Opts), ctypes.sizeof(Stats)):
        raise RuntimeError("libeik struct sizes %d/%d differ from the binding's %d/%d: "
                           "rebuild the library" % (so.value, ss.value, ctypes.sizeof(Opts),
                                                    ctypes.sizeof(Stats)))
    if path == LIB_PATH or _lib is None:
        _lib = lib
    return lib


def selftest_local_solve(count=1 << 22, seed=1, device=0):
    """Largest difference between the sweeps' FP64 local solve and the
    direct FP64 closed forms over `count` random inputs: (in ulps of the
    direct result, in units of ulp + 2^-44 s)."""
    mu, mr = ctypes.c_double(), ctypes.c_double()
    rc = load().eik_selftest_local_solve(int(device), int(count), int(seed), ctypes.byref(mu),
                                         ctypes.byref(mr))
    if rc != 0:
        raise EikError(rc, "eik_selftest_local_solve")
    return mu.value, mr.value


def default_opts() -> Opts:
    o = Opts()
    load().eik_opts_default(ctypes.byref(o))
    return o


def make_opts(precision="fp32_polish", cell_n=0, device=0, hbm_budget_bytes=0,
              spin_cap_us=None, bucket_width=None, max_sweeps_per_visit=None, max_ctas=0,
              bulk_kappa_rel=None, queue_order=None, use_graphs=None,
              cell_key=None, serve_batch_nodes=None, polish_lift=None,
              warps_per_cell=None) -> Opts:
    """eik_opts from the library defaults with the given fields changed
    (None = keep the default)."""
    o = default_opts()
    o.device = int(device)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.cell_n = int(cell_n)
    o.max_ctas = int(max_ctas)
    o.hbm_budget_bytes = int(hbm_budget_bytes)
    if spin_cap_us is not None:
        o.spin_cap_us = int(spin_cap_us)
    if bucket_width is not None:
        o.bucket_width = float(bucket_width)
    if max_sweeps_per_visit is not None:
        o.max_sweeps_per_visit = int(max_sweeps_per_visit)
    if bulk_kappa_rel is not None:
        o.bulk_kappa_rel = float(bulk_kappa_rel)
    if queue_order is not None:
        o.queue_order = int(queue_order)
    if use_graphs is not None:
        o.use_graphs = int(use_graphs)
    if cell_key is not None:
        o.cell_key = int(cell_key)
    if serve_batch_nodes is not None:
        o.serve_batch_nodes = int(serve_batch_nodes)
    if polish_lift is not None:
        o.polish_lift = float(polish_lift)
    if warps_per_cell is not None:
        o.warps_per_cell = int(warps_per_cell)
    return o


def _host_arrays(F, mask, q):
    F = np.ascontiguousarray(F, dtype=np.float32)
    if F.ndim != 3:
        raise ValueError("F must have shape (nz, ny, nx)")
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    q = np.ascontiguousarray(q, dtype=np.float64)
    if mask.shape != F.shape or q.shape != F.shape:
        raise ValueError("F, mask and q must have one shape")
    return F, mask, q


def _dims_of(shape):
    nz, ny, nx = shape
    return (ctypes.c_int64 * 3)(nx, ny, nz)


def _is_torch_cuda(x):
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


class Solver:
    """One eik_ctx: device memory and options for a sequence of solves."""

    def __init__(self, precision="fp32_polish", cell_n=0, device=0,
                 hbm_budget_bytes=0, spin_cap_us=None, bucket_width=None,
                 max_sweeps_per_visit=None, max_ctas=0, bulk_kappa_rel=None,
                 queue_order=None, use_graphs=None, cell_key=None, serve_batch_nodes=None,
                 polish_lift=None, warps_per_cell=None):
        """Options left at None keep the library defaults (eik_opts_default)."""
        self.lib = load()
        o = make_opts(precision=precision, cell_n=cell_n, device=device,
                      hbm_budget_bytes=hbm_budget_bytes, spin_cap_us=spin_cap_us,
                      bucket_width=bucket_width, max_sweeps_per_visit=max_sweeps_per_visit,
                      max_ctas=max_ctas, bulk_kappa_rel=bulk_kappa_rel,
                      queue_order=queue_order, use_graphs=use_graphs, cell_key=cell_key,
                      serve_batch_nodes=serve_batch_nodes, polish_lift=polish_lift,
                      warps_per_cell=warps_per_cell)
        self.opts = o
        self._outputs = {}  # ticket -> output array, alive until done or cancelled
        self.ctx = ctypes.c_void_p()
        rc = self.lib.eik_create(ctypes.byref(self.ctx), ctypes.byref(o))
        if rc != EIK_OK:
            raise EikError(rc, "eik_create")

    def close(self):
        if self.ctx:
            self.lib.eik_destroy(self.ctx)  # waits for batches still on the device
            self.ctx = ctypes.c_void_p()
            self._outputs.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- one grid ---------------------------------------------------------
    def solve(self, F, mask, q, h, tol=0.0, out=None, stream=None, check=True):
        """Solve one grid.  numpy inputs -> eik_solve (host buffers, numpy
        result; page-locked buffers, e.g. the .numpy() views of pinned torch
        tensors, are read and written in place by the device instead of
        copied); torch CUDA tensors -> eik_solve_device (result tensor).
        Returns (u, stats_dict)."""
        st = Stats()
        if _is_torch_cuda(F):
            import torch
            F_t = F.contiguous()
            m_t = mask.contiguous()
            q_t = q.contiguous()
            if F_t.dtype != torch.float32 or m_t.dtype != torch.uint8 or q_t.dtype != torch.float64:
                raise TypeError("device inputs must be float32 F, uint8 mask, float64 q")
            u = out if out is not None else torch.empty(F_t.shape, dtype=torch.float64,
                                                        device=F_t.device)
            s = stream if stream is not None else torch.cuda.current_stream(F_t.device).cuda_stream
            rc = self.lib.eik_solve_device(self.ctx, _dims_of(F_t.shape), float(h),
                                           F_t.data_ptr(), m_t.data_ptr(), q_t.data_ptr(),
                                           float(tol), u.data_ptr(), ctypes.c_void_p(s),
                                           ctypes.byref(st))
        else:
            F_h, m_h, q_h = _host_arrays(F, mask, q)
            u = out if out is not None else np.empty(F_h.shape, dtype=np.float64)
            rc = self.lib.eik_solve(self.ctx, _dims_of(F_h.shape), float(h),
                                    F_h.ctypes.data, m_h.ctypes.data, q_h.ctypes.data,
                                    float(tol), u.ctypes.data, ctypes.byref(st))
        if rc != EIK_OK and check:
            raise EikError(rc, "eik_solve")
        d = st.as_dict()
        d["status"] = rc
        return u, d

    def autotune(self, F, mask, q, h, tol=0.0):
        """Pick cell size and cell-kernel CTAs for grids of this size
        (eik_autotune); returns (cell_n, ctas)."""
        F_h, m_h, q_h = _host_arrays(F, mask, q)
        bn, bc = ctypes.c_int(0), ctypes.c_int(0)
        rc = self.lib.eik_autotune(self.ctx, _dims_of(F_h.shape), float(h), F_h.ctypes.data,
                                   m_h.ctypes.data, q_h.ctypes.data, float(tol),
                                   ctypes.byref(bn), ctypes.byref(bc))
        if rc != EIK_OK:
            raise EikError(rc, "eik_autotune")
        return bn.value, bc.value

    # -- many grids in one launch -------------------------------------------
    def solve_batch(self, problems, tol=0.0, check=True):
        """problems: list of (F, mask, q, h) numpy tuples.  Returns (list of u, stats)."""
        count = len(problems)
        arrs = [_host_arrays(F, m, q) for (F, m, q, _) in problems]
        dims = (ctypes.c_int64 * (3 * count))()
        for t, (F, _, _) in enumerate(arrs):
            nz, ny, nx = F.shape
            dims[3 * t:3 * t + 3] = [nx, ny, nz]
        hs = (ctypes.c_double * count)(*[float(p[3]) for p in problems])
        outs = [np.empty(a[0].shape, dtype=np.float64) for a in arrs]
        VP = ctypes.c_void_p * count
        st = Stats()
        rc = self.lib.eik_solve_batch(self.ctx, count, dims, hs,
                                      VP(*[a[0].ctypes.data for a in arrs]),
                                      VP(*[a[1].ctypes.data for a in arrs]),
                                      VP(*[a[2].ctypes.data for a in arrs]),
                                      float(tol), VP(*[o.ctypes.data for o in outs]),
                                      ctypes.byref(st))
        if rc != EIK_OK and check:
            raise EikError(rc, "eik_solve_batch")
        d = st.as_dict()
        d["status"] = rc
        return outs, d

    def solve_batch_device(self, problems, tol=0.0, outs=None, stream=None, check=True):
        """problems: list of (F, mask, q, h) with torch CUDA tensors."""
        import torch
        count = len(problems)
        dims = (ctypes.c_int64 * (3 * count))()
        for t, (F, _, _, _) in enumerate(problems):
            nz, ny, nx = F.shape
            dims[3 * t:3 * t + 3] = [nx, ny, nz]
        hs = (ctypes.c_double * count)(*[float(p[3]) for p in problems])
        if outs is None:
            outs = [torch.empty(p[0].shape, dtype=torch.float64, device=p[0].device)
                    for p in problems]
        VP = ctypes.c_void_p * count
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        st = Stats()
        rc = self.lib.eik_solve_batch_device(
            self.ctx, count, dims, hs, VP(*[p[0].data_ptr() for p in problems]),
            VP(*[p[1].data_ptr() for p in problems]), VP(*[p[2].data_ptr() for p in problems]),
            float(tol), VP(*[o.data_ptr() for o in outs]), ctypes.c_void_p(s), ctypes.byref(st))
        if rc != EIK_OK and check:
            raise EikError(rc, "eik_solve_batch_device")
        d = st.as_dict()
        d["status"] = rc
        return outs, d

    # -- serving ------------------------------------------------------------
    def submit(self, F, mask, q, h, tol=0.0, out=None):
        """Queue one solve; returns (ticket, out array filled on completion).
        The binding keeps the input and output arrays alive until the ticket
        is done or cancelled (the library uses them asynchronously).  A
        page-locked `out` is written in place by the device; cancelling such
        a request while it runs waits for its batch."""
        F_h, m_h, q_h = _host_arrays(F, mask, q)
        u = out if out is not None else np.empty(F_h.shape, dtype=np.float64)
        if not (u.flags.c_contiguous and u.dtype == np.float64 and u.shape == F_h.shape):
            raise ValueError("out must be a C-contiguous float64 array of F's shape")
        t = ctypes.c_uint64()
        rc = self.lib.eik_submit(self.ctx, _dims_of(F_h.shape), float(h), F_h.ctypes.data,
                                 m_h.ctypes.data, q_h.ctypes.data, float(tol), u.ctypes.data,
                                 ctypes.byref(t))
        if rc != EIK_OK:
            raise EikError(rc, "eik_submit")
        # the library reads the inputs and writes u until the ticket is done
        self._outputs[t.value] = (u, F_h, m_h, q_h)
        return t.value, u

    def poll(self, ticket):
        """Returns (done, status, stats_dict)."""
        done = ctypes.c_int(0)
        st = Stats()
        rc = self.lib.eik_poll(self.ctx, ctypes.c_uint64(ticket), ctypes.byref(done),
                               ctypes.byref(st))
        if done.value:
            self._outputs.pop(ticket, None)
        return bool(done.value), rc, st.as_dict()

    def cancel(self, ticket):
        rc = self.lib.eik_cancel(self.ctx, ctypes.c_uint64(ticket))
        if rc == EIK_OK:
            self._outputs.pop(ticket, None)
        return rc


def solve(F, mask, q, h, tol=0.0, precision="fp32_polish", cell_n=0):
    """One-shot convenience wrapper: returns u (numpy or torch, like F)."""
    with Solver(precision=precision, cell_n=cell_n) as s:
        u, _ = s.solve(F, mask, q, h, tol)
    return u


def dfsm_solve(F, mask, q, h, tol=0.0, max_sweeps=4096, out=None, stream=None, check=True):
    """Whole-grid sweeping baseline (eik_dfsm_solve_device) on torch CUDA
    tensors F (float32), mask (uint8), q (float64), shape (nz, ny, nx).
    Returns (u, stats_dict) with the per-sweep counts and largest decreases
    in stats_dict["changed_per_sweep"] / ["max_drop_per_sweep"]."""
    import torch
    if not (_is_torch_cuda(F) and _is_torch_cuda(mask) and _is_torch_cuda(q)):
        raise TypeError("dfsm_solve takes torch CUDA tensors")
    F_t, m_t, q_t = F.contiguous(), mask.contiguous(), q.contiguous()
    if F_t.dtype != torch.float32 or m_t.dtype != torch.uint8 or q_t.dtype != torch.float64:
        raise TypeError("device inputs must be float32 F, uint8 mask, float64 q")
    u = out if out is not None else torch.empty(F_t.shape, dtype=torch.float64, device=F_t.device)
    s = stream if stream is not None else torch.cuda.current_stream(F_t.device).cuda_stream
    nsw = ctypes.c_int64(0)
    chg = (ctypes.c_int64 * int(max_sweeps))()
    drop = (ctypes.c_double * int(max_sweeps))()
    st = Stats()
    with torch.cuda.device(F_t.device):
        rc = load().eik_dfsm_solve_device(_dims_of(F_t.shape), float(h), F_t.data_ptr(),
                                          m_t.data_ptr(), q_t.data_ptr(), float(tol),
                                          int(max_sweeps), u.data_ptr(), ctypes.c_void_p(s),
                                          ctypes.byref(nsw), chg, drop, ctypes.byref(st))
    if rc != EIK_OK and check:
        raise EikError(rc, "eik_dfsm_solve_device")
    d = st.as_dict()
    d["status"] = rc
    d["changed_per_sweep"] = [int(chg[k]) for k in range(nsw.value)]
    d["max_drop_per_sweep"] = [float(drop[k]) for k in range(nsw.value)]
    return u, d
