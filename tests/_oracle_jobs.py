"""Oracle FMM solves of the large workloads, run in the background during a
GPU test session (test infrastructure).

A test that needs the FMM solution of a large workload carries the marker
``fmm_solution(name, arg)``.  When the session's selected tests include any
such test and a CUDA device is present, ``start`` submits every marked
workload to a pool of spawned oracle workers right after collection
(oracle/fmm_cache.py), so the minutes of serial FMM overlap the GPU tests
that run first; ``solution`` waits for one result.  Without a GPU nothing is
started (the marked tests skip).
"""
import concurrent.futures as cf

_pool = None
_futs = {}


def start(tasks):
    global _pool
    from oracle import fmm_cache
    if not tasks:
        return
    # the 513^3 solve is the long pole: submit the largest first
    tasks = sorted(set(tasks), key=lambda t: (t[0] != "barrier", t[1]))
    _pool = fmm_cache.make_pool()
    for t in tasks:
        _futs[t] = _pool.submit(fmm_cache.solve_named, *t)


def solution(name, arg, timeout=900):
    """The FMM solution (read-only memory map) of a started workload, or of
    one solved here on demand when it was not started."""
    from oracle import fmm_cache
    f = _futs.get((name, arg))
    if f is None:
        path, _ = fmm_cache.solve_named(name, arg)
    else:
        path, _ = f.result(timeout=timeout)
    return fmm_cache.load(path)


def stop():
    global _pool
    if _pool is None:
        return
    for f in _futs.values():
        f.cancel()
    procs = list(getattr(_pool, "_processes", {}).values())
    _pool.shutdown(wait=False, cancel_futures=True)
    for p in procs:  # our own workers, by their process objects
        if p.is_alive():
            p.terminate()
    _pool = None
    _futs.clear()
