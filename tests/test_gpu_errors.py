"""Failure paths of the product on the GPU, driven through the C ABI without
any fault: a Jacobi SVD sweep cap that the wide merges cannot meet must make
h2_mul return H2_ENOCONV (the kernels stop at the cap and set the error flag;
nothing waits or traps), and the library must stay usable afterwards."""
import numpy as np
import pytest

from paper_2403_01566_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2403_01566_gb300 import h2  # noqa: E402


def test_svd_sweep_cap_returns_enoconv_and_recovers():
    w = I.grid_2d(32, 1e-6)
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
    with pytest.raises(h2.H2Error) as ei:
        h2.mul(A, B, w.eps, svd_max_sweeps=1)
    assert ei.value.code == h2.H2_ENOCONV
    # the same cached plan with the default cap: a normal product
    C1 = h2.mul(A, B, w.eps)
    C2 = h2.mul(A, B, w.eps, svd_max_sweeps=60)
    x = I.random_vector(w.n, 5)
    y1, y2 = C1.matvec(x), C2.matvec(x)
    assert np.array_equal(y1, y2)
    ref = A.matvec(B.matvec(x))
    assert np.linalg.norm(y1 - ref) <= 1e-5 * np.linalg.norm(ref)
