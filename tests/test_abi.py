"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point declared in include/h2.h; argument validation
happens before any device work."""
import ctypes as C
import os

import numpy as np
import pytest

import __graft_entry__ as G
from paper_2403_01566_gb300 import h2


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(h2.LIB_PATH):
        G.build()
    return h2._lib()


def test_exports_every_declared_symbol(lib):
    names = h2.exported_symbols()
    assert {"h2_build", "h2_mul", "h2_matvec", "h2_free"} <= set(names)
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/h2.h but not exported"


def test_strerror_codes(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.h2_strerror(code)
    assert lib.h2_strerror(-7).decode().startswith("adaptive rank")
    assert "did not converge" in lib.h2_strerror(h2.H2_ENOCONV).decode()
    assert "timed out" in lib.h2_strerror(h2.H2_ETIMEOUT).decode()


def test_build_rejects_invalid_arguments(lib):
    pts = np.zeros((4, 2))
    o = h2.BuildOpts()
    o.eta, o.leaf_size, o.order, o.kernel, o.dim = 2.0, 32, 4, 0, 2
    out = C.c_void_p()
    dp = C.POINTER(C.c_double)
    assert lib.h2_build(pts.ctypes.data_as(dp), 0, C.byref(o), C.byref(out)) == h2.H2_EINVAL
    o.dim = 4
    assert lib.h2_build(pts.ctypes.data_as(dp), 4, C.byref(o), C.byref(out)) == h2.H2_EINVAL
    o.dim, o.leaf_size = 2, 1
    assert lib.h2_build(pts.ctypes.data_as(dp), 4, C.byref(o), C.byref(out)) == h2.H2_EINVAL
    o.leaf_size = 32
    bad = np.array([[0.0, np.nan], [1.0, 1.0]])
    assert lib.h2_build(bad.ctypes.data_as(dp), 2, C.byref(o), C.byref(out)) == h2.H2_EINVAL
    assert out.value is None


def test_mul_rejects_null_handles(lib):
    out = C.c_void_p()
    assert lib.h2_mul(None, None, C.c_double(1e-6), None, C.byref(out)) == h2.H2_EINVAL
