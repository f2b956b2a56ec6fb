"""h2_matvec_noalloc: the allocation-free matrix-vector product (for callers
that cannot call cudaMalloc: loops that must stay out of the allocator, or
processes whose device memory is partitioned up front) must give the same y
as h2_matvec, call after call.  Its scratch is a static device array shared
by all calls, so two calls in a row must not see each other's leftovers.
This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2403_01566_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2403_01566_gb300 import h2  # noqa: E402


def _noalloc(M, x_cluster):
    lib = h2._lib()
    lib.h2_matvec_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    x = torch.tensor(x_cluster, dtype=torch.float64, device="cuda")
    y = torch.full_like(x, float("nan"))
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.h2_matvec_noalloc(M.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), C.c_void_p(stream))
    assert rc == 0, h2._lib().h2_strerror(rc)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("w", [I.plain_1d(1024), I.grid_2d(32)], ids=lambda w: w.name)
def test_noalloc_matvec_matches_h2_matvec(w):
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
    C_ = h2.mul(A, B, 1e-6)           # a product: adaptive ranks, padded storage
    for M in (A, C_):
        perm = M.permutation()
        for call in range(2):          # two calls in a row share the static scratch
            x = I.random_vector(w.n, 100 + call)
            y_ref = M.matvec(x)        # existing entry point, caller ordering
            y = _noalloc(M, x[perm])   # cluster ordering
            ref = y_ref[perm]
            assert np.all(np.isfinite(y))
            assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)


def test_noalloc_rejects_trees_beyond_its_scratch():
    """A matrix whose coefficient vectors (2 * nclusters * kpad doubles) do not
    fit the fixed 2^20-double scratch is refused with H2_ENOMEM before any
    device work: 1D, order 8 (k = 8), leaf 2, n = 131072 has 131071 clusters."""
    n = 131072
    pts = I.uniform_points(n, 1, 77)
    M = h2.build(pts, I.LOG, 2.0, 2, 8)
    st = M.info()
    assert 2 * st.nclusters * st.kpad > (1 << 20)
    lib = h2._lib()
    lib.h2_matvec_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    rc = lib.h2_matvec_noalloc(M.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), None)
    assert rc == h2.H2_ENOMEM


def test_noalloc_rejects_host_vectors():
    """x and y must be device memory of the current device."""
    w = I.plain_1d(256)
    M = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    lib = h2._lib()
    lib.h2_matvec_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    xh = np.zeros(w.n)
    yd = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    rc = lib.h2_matvec_noalloc(M.handle, C.c_void_p(xh.ctypes.data), C.c_void_p(yd.data_ptr()), None)
    assert rc == h2.H2_EINVAL
