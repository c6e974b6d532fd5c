"""FMM solutions of the large seeded workloads, computed by the oracle only
and kept in a file cache (test infrastructure).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
``cpu_baseline`` / reference legs may use this module.  It calls nothing but
``oracle`` (the serial FP64 FMM of oracle.c) and the seeded input
generators of ``paper_1306_4743_gb300.workloads``, which hold none of the
solver's arithmetic; no value here ever comes from the CUDA library.

A full FMM of the 513^3 barrier field (135 M nodes) takes about two minutes
on one core, and the 256 instances of the batch workload about a minute and
a half in all, so the solutions are

* keyed by a SHA-256 digest of the inputs (F, mask, q, h and the shape), so a
  cached file can only be reused for bit-identical inputs;
* stored as ``<digest>.npy`` under ``$EIK_ORACLE_CACHE`` or
  ``oracle/_cache`` (kept out of version control and of the GPU-box copy);
* computed in worker processes started with ``spawn`` (never forked from a
  process that may hold a CUDA context), one problem per worker, so the
  batch instances run in parallel and the 513^3 solve overlaps them.

Workers regenerate their problem from its recipe name instead of receiving
gigabytes of input through a pipe.

    python -m oracle.fmm_cache [--jobs N] [barrier513] [batch256]

fills the cache for the named workloads and prints the time of each solve.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import multiprocessing
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def cache_dir() -> str:
    d = os.environ.get("EIK_ORACLE_CACHE") or os.path.join(HERE, "_cache")
    os.makedirs(d, exist_ok=True)
    return d


def digest(p) -> str:
    """SHA-256 of a problem's inputs (shape, h, F, mask, q)."""
    h = hashlib.sha256()
    h.update(repr((tuple(p.F.shape), float(p.h))).encode())
    for a in (p.F, p.mask, p.q):
        h.update(np.ascontiguousarray(a).view(np.uint8).reshape(-1).data)
    return h.hexdigest()[:32]


def problem(name: str, arg: int, n_requests: int = 500):
    """The seeded workload `name` with parameter `arg`:
    ("barrier", m) the barrier-block field on m^3 nodes (16 boxes a side,
    p = 0.3, F = 0.01, 8 exits); ("osc", m) the oscillatory speed
    1 + 0.5 sin(4 pi x) sin(4 pi y) sin(4 pi z) on m^3 nodes; ("point", m) the
    F = 1 point source on m^3 nodes; ("batch", k) instance k of the 256-instance
    batch; ("serve", k) request k of the serving stream of `n_requests`
    draws (the edges depend on the stream length)."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_1306_4743_gb300 import workloads as W
    if name == "barrier":
        return W.barrier_blocks(arg)
    if name == "osc":
        return W.oscillatory(arg)
    if name == "point":
        return W.point_source_const(arg)
    if name == "batch":
        return W.gaussian_bumps(W.batch_dims(arg + 1)[arg], 4000 + arg)
    if name == "serve":
        _, edge, seed = W.serving_requests(n=n_requests, rate=1.0, seed=5)[arg]
        return W.serving_problem(edge, seed)
    raise ValueError("unknown workload " + name)


def cached_fmm(p, mmap: bool = True, force: bool = False):
    """u = orc_fmm(p) from the cache, computing and storing it on a miss (or
    always, with force, so that the solve is timed).  Returns (u, seconds of
    the FMM solve or None when it came from the cache)."""
    import oracle
    path = os.path.join(cache_dir(), digest(p) + ".npy")
    if os.path.exists(path) and not force:
        return np.load(path, mmap_mode="r" if mmap else None), None
    t0 = time.perf_counter()
    u = oracle.fmm(p.F, p.mask, p.q, p.h)
    dt = time.perf_counter() - t0
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "wb") as f:
        np.save(f, u)
    os.replace(tmp, path)
    return u, dt


def solve_named(name: str, arg: int, n_requests: int = 500, force: bool = False):
    """Worker entry: regenerate the problem, take its FMM solution from the
    cache or compute it (always with force).  Returns (cache path, FMM
    seconds or None when it came from the cache)."""
    p = problem(name, arg, n_requests)
    path = os.path.join(cache_dir(), digest(p) + ".npy")
    _, dt = cached_fmm(p, force=force)
    return path, dt


def make_pool(jobs: int | None = None) -> cf.ProcessPoolExecutor:
    """A pool of oracle worker processes started with spawn."""
    from .build import build_oracle
    build_oracle()  # once, before workers load it
    if jobs is None:
        jobs = max(1, min(12, (os.cpu_count() or 2) - 2))
    return cf.ProcessPoolExecutor(max_workers=jobs,
                                  mp_context=multiprocessing.get_context("spawn"))


def load(path: str):
    return np.load(path, mmap_mode="r")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("which", nargs="*", default=["barrier513", "batch256"])
    a = ap.parse_args(argv)
    tasks = []
    if "barrier513" in a.which:
        tasks.append(("barrier", 513))
    if "batch256" in a.which:
        tasks += [("batch", k) for k in range(256)]
    t0 = time.perf_counter()
    with make_pool(a.jobs) as pool:
        futs = {pool.submit(solve_named, n, k): (n, k) for (n, k) in tasks}
        for f in cf.as_completed(futs):
            path, dt = f.result()
            n, k = futs[f]
            print("%s %d: %s (%s)" % (n, k, os.path.basename(path),
                                      "cached" if dt is None else "%.1f s" % dt))
    print("done in %.1f s" % (time.perf_counter() - t0))


if __name__ == "__main__":
    main()
