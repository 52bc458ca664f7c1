"""The C ABI without a GPU: the library loads, exports every function that
include/h2mg.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "h2mg.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2501_17656_gb300 import _build
    import paper_2501_17656_gb300 as pkg
    _build.build()
    return pkg.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(h2mg_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "h2mg_build" in names and "h2mg_solve" in names and "h2mg_apply" in names
    for name in names:
        assert hasattr(lib, name), name
    import paper_2501_17656_gb300 as pkg
    assert set(pkg.EXPORTED) <= set(names)


def test_error_strings(lib):
    for s in range(9):
        assert lib.h2mg_error_string(s).decode()
    assert lib.h2mg_error_string(99).decode() == "unknown status"


def test_build_rejects_bad_arguments_without_cuda(lib):
    import paper_2501_17656_gb300 as pkg
    pts = np.random.default_rng(0).random((100, 2))
    h = ctypes.c_void_p()
    k = pkg._Kernel(0, 0.1, 0.0, 2, None, None)
    good = pkg._BuildOpts(32, 3, 1.0, 0, 0, -1)
    cases = [
        (None, 100, 2, k, good),                                     # null points
        (pts.ctypes.data, 0, 2, k, good),                            # n < 1
        (pts.ctypes.data, 100, 4, k, good),                          # dim
        (pts.ctypes.data, 100, 2, k, pkg._BuildOpts(1, 3, 1.0, 0, 0, -1)),    # leaf
        (pts.ctypes.data, 100, 2, k, pkg._BuildOpts(32, 9, 1.0, 0, 0, -1)),   # rank 81 > 64
        (pts.ctypes.data, 100, 2, k, pkg._BuildOpts(32, 3, -1.0, 0, 0, -1)),  # eta
        (pts.ctypes.data, 100, 2, k, pkg._BuildOpts(32, 3, 1.0, 7, 0, -1)),   # storage
        (pts.ctypes.data, 100, 2, pkg._Kernel(0, -0.1, 0.0, 2, None, None), good),  # length
        (pts.ctypes.data, 100, 2, pkg._Kernel(3, 1.0, 0.0, 2, None, None), good),   # single layer without areas or diagonal
        (pts.ctypes.data, 100, 2, pkg._Kernel(9, 1.0, 0.0, 2, None, None), good),   # kind
        (pts.ctypes.data, 100, 2, k, pkg._BuildOpts(32, 3, 1.0, 0, 0, -1, 2, 1e-9, 64)),   # basis kind
        (pts.ctypes.data, 100, 2, k, pkg._BuildOpts(32, 3, 1.0, 0, 0, -1, 1, 1e-9, 0)),    # skeleton rank 0
        (pts.ctypes.data, 100, 2, k, pkg._BuildOpts(32, 3, 1.0, 0, 0, -1, 1, 1e-9, 65)),   # skeleton rank > 64
        (pts.ctypes.data, 100, 2, k, pkg._BuildOpts(32, 3, 1.0, 0, 0, -1, 1, -1.0, 64)),   # negative tolerance
    ]
    for (p, n, d, kk, o) in cases:
        st = lib.h2mg_build(p, n, d, ctypes.byref(kk), ctypes.byref(o), None, ctypes.byref(h))
        assert st in (1, 8), st
        assert not h.value
        assert lib.h2mg_last_error().decode()


def test_null_handles(lib):
    assert lib.h2mg_destroy(None) == 0
    v = ctypes.c_int64()
    assert lib.h2mg_query(None, 0, 0, ctypes.byref(v)) == 1
    assert lib.h2mg_apply(None, None, None, 1, 1, None) == 1
    assert lib.h2mg_apply_noalloc(None, None, None, None) == 1
    assert lib.h2mg_profile(None, 1, None, None, None) == 1
    assert lib.h2mg_autotune(None, None, None, 0, None) == 1
    out = ctypes.c_double()
    assert lib.h2mg_dot(None, None, 4, ctypes.byref(out), None) == 1
    import paper_2501_17656_gb300 as pkg
    k = pkg._Kernel(5, 0.1, 0.0, 2, None, None)
    h = ctypes.c_void_p()
    assert lib.h2mg_build_sibling(None, ctypes.byref(k), None, ctypes.byref(h)) == 1 and not h.value


def test_batched_solve_rejects_bad_arguments_without_cuda(lib):
    import paper_2501_17656_gb300 as pkg
    o = pkg.H2Matrix._opts()
    infos = (pkg.SolveInfo * 2)()
    arr = ctypes.c_void_p * 2
    nul = arr(None, None)
    assert lib.h2mg_solve_batched(0, nul, nul, nul, ctypes.byref(o), infos, None) == 1      # no problems
    assert lib.h2mg_solve_batched(2, None, nul, nul, ctypes.byref(o), infos, None) == 1     # null list
    assert lib.h2mg_solve_batched(2, nul, nul, nul, ctypes.byref(o), infos, None) == 1      # null handles
    bad = pkg.H2Matrix._opts(max_cycles=-1)
    assert lib.h2mg_solve_batched(2, nul, nul, nul, ctypes.byref(bad), infos, None) == 1
    assert lib.h2mg_last_error().decode()



def test_solve_rejects_bad_outer_and_cycle_without_cuda(lib):
    """An unknown outer loop or cycle type is refused (here with a null handle the
    handle check comes first; the batched solve checks its options before the
    handles)."""
    import paper_2501_17656_gb300 as pkg
    infos = (pkg.SolveInfo * 2)()
    arr = ctypes.c_void_p * 2
    nul = arr(None, None)
    for field, val in (("outer", 2), ("outer", 9), ("cycle", 3), ("cycle", -1)):
        o = pkg.H2Matrix._opts()
        setattr(o, field, val)
        assert lib.h2mg_solve_batched(2, nul, nul, nul, ctypes.byref(o), infos, None) == 1
        assert lib.h2mg_last_error().decode()
