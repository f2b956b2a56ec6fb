"""The precision workload at its full size: n = 65536 Fibonacci points on the
sphere, A = 1/(4 pi |x-y|) (diag 0), leaf 64, eta 2, order 4 (k = 64),
C = A*A at eps = 1e-6 (178 GB of workspace on one GB300).

The oracle cannot run this size, so the test checks properties that hold at
any size:
- C x against A (A x) through the H^2 matrix-vector product (itself checked
  against the oracle's) within the block bound eps, summed over the blocks of
  a row: eps sqrt(2 * 64) relative;
- the compensated form (precision 2) against the FP64 form: the same ranks
  and C x within 1e-10 relative (both are FP64-accurate)."""
import numpy as np
import pytest

from paper_2403_01566_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900, method="thread")]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2403_01566_gb300 import h2  # noqa: E402


def test_sphere_65536_k64_bound_and_forms_agree():
    w = I.sphere_3d(65536, 1e-6)
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    xs = [I.random_vector(w.n, s) for s in (1, 2)]
    C = h2.mul(A, A, w.eps)
    y64 = [C.matvec(x) for x in xs]
    rr64, rc64 = C.ranks()
    C.free()
    Cdf = h2.mul(A, A, w.eps, precision=2)
    ydf = [Cdf.matvec(x) for x in xs]
    rrdf, rcdf = Cdf.ranks()
    Cdf.free()
    assert list(rr64) == list(rrdf) and list(rc64) == list(rcdf)
    for x, a, b in zip(xs, y64, ydf):
        z = A.matvec(A.matvec(x))
        assert np.linalg.norm(a - z) <= w.eps * np.sqrt(2 * 64) * np.linalg.norm(z)
        assert np.linalg.norm(b - a) <= 1e-10 * np.linalg.norm(a)
