"""The C ABI library builds for sm_103a, loads, and exports every entry
point that include/eik.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "eik.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eik_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("eik_create", "eik_solve", "eik_destroy", "eik_submit", "eik_poll",
                     "eik_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1306_4743_gb300 import eik
    lib = eik.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(eik.EXPORTED) == declared_functions()


def test_defaults_and_strerror_without_gpu():
    from paper_1306_4743_gb300 import eik
    o = eik.default_opts()
    assert o.precision == 1 and o.cell_n == 0 and o.spin_cap_us == 5_000_000
    assert o.max_sweeps_per_visit == 4096 and o.bucket_width == 0.25 and o.queue_order == 1
    lib = eik.load()
    assert lib.eik_strerror(0) == b"ok"
    assert lib.eik_strerror(5).startswith(b"device wait")
    assert lib.eik_strerror(12345) == b"unknown status"


def test_struct_mirrors_match_the_library():
    from paper_1306_4743_gb300 import eik
    lib = eik.load()
    so, ss = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.eik_struct_sizes(ctypes.byref(so), ctypes.byref(ss)) == 0
    assert so.value == ctypes.sizeof(eik.Opts) and ss.value == ctypes.sizeof(eik.Stats)
    assert lib.eik_struct_sizes(None, None) == 0


def test_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1306_4743_gb300 import eik
    with pytest.raises(eik.EikError) as e:
        eik.Solver()
    assert e.value.status == 4  # EIK_ECUDA, not a crash


def test_invalid_options_rejected_before_device_use():
    from paper_1306_4743_gb300 import eik
    lib = eik.load()
    o = eik.default_opts()
    o.cell_n = 5
    ctx = ctypes.c_void_p()
    assert lib.eik_create(ctypes.byref(ctx), ctypes.byref(o)) == 1
    o = eik.default_opts()
    o.precision = 7
    assert lib.eik_create(ctypes.byref(ctx), ctypes.byref(o)) == 1
    o = eik.default_opts()
    o.cell_key = 2
    assert lib.eik_create(ctypes.byref(ctx), ctypes.byref(o)) == 1
    o = eik.default_opts()
    o.warps_per_cell = 5
    assert lib.eik_create(ctypes.byref(ctx), ctypes.byref(o)) == 1
    o = eik.default_opts()
    o.polish_lift = -0.75  # would start the polish far below any fixed point
    assert lib.eik_create(ctypes.byref(ctx), ctypes.byref(o)) == 1
    assert not ctx


def test_binding_keeps_library_defaults():
    from paper_1306_4743_gb300 import eik
    d = eik.default_opts()
    o = eik.make_opts()
    for name, _ in eik.Opts._fields_:
        assert getattr(o, name) == getattr(d, name), name
    o = eik.make_opts(precision="fp64", cell_n=16, queue_order=0, bucket_width=2.0)
    assert (o.precision, o.cell_n, o.queue_order, o.bucket_width) == (0, 16, 0, 2.0)
    assert o.bulk_kappa_rel == d.bulk_kappa_rel and o.spin_cap_us == d.spin_cap_us


def test_oversized_grids_rejected_before_any_product_overflows():
    """Edges up to 2^24 each would give up to 2^72 nodes: the entry points
    must bound the node count before forming it, and return before any
    device call.  Dummy (non-null) pointers are never dereferenced."""
    from paper_1306_4743_gb300 import eik
    lib = eik.load()
    dummy = ctypes.c_void_p(16)
    for d in ((1 << 24, 1 << 24, 1 << 24), (1 << 24, 1 << 24, 2), (400, 400, 400),
              (1 << 23, 1, 1)):
        dims = (ctypes.c_int64 * 3)(*d)
        rc = lib.eik_solve_device_noalloc(dims, 0.01, dummy, dummy, dummy, 0.0, dummy, None,
                                          None)
        assert rc == 3, (d, rc)  # EIK_EBUDGET: cannot fit the fixed scratch
    dims = (ctypes.c_int64 * 3)(1 << 25, 1, 1)
    assert lib.eik_solve_device_noalloc(dims, 0.01, dummy, dummy, dummy, 0.0, dummy, None,
                                        None) == 1  # edge above 2^24: EIK_EINVAL
