"""Batched H^2 matrix-vector products (many right-hand sides) against the
dense matrix and the oracle's matrix-vector product, for input matrices and
for a product C; host and device operands; edge cases (one column, a column
count that spans several 64-column tiles with a ragged tail, the maximum)."""
import numpy as np
import pytest

from oracle import h2oracle as O
from paper_2403_01566_gb300 import inputs as I
from tests.oracle_cases import build_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2403_01566_gb300 import h2  # noqa: E402


def _rel(a, b):
    return np.linalg.norm(a - b) / (np.linalg.norm(b) or 1.0)


@pytest.mark.parametrize("nrhs", [1, 7, 64, 130])
def test_batch_matches_dense_and_oracle(nrhs):
    w = I.grid_2d(32)
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    X = np.random.default_rng(nrhs).standard_normal((w.n, nrhs))
    Y = A.matvec_batch(X)
    Ad = A.to_dense()
    assert _rel(Y, Ad @ X) <= 1e-13
    Xo, _ = build_pair(w)
    Yo = np.stack([Xo.matvec(X[:, j]) for j in range(nrhs)], axis=1)
    assert _rel(Y, Yo) <= 1e-13
    # single-vector entry point agrees column by column
    assert _rel(A.matvec(X[:, 0]), Y[:, 0]) <= 1e-15


def test_batch_device_operands_and_product_matrix():
    w = I.grid_2d(32)
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
    C = h2.mul(A, B, 1e-6)
    X = np.random.default_rng(3).standard_normal((w.n, 33))
    Yd = C.matvec_batch(torch.from_numpy(X).cuda()).cpu().numpy()
    Yh = C.matvec_batch(X)
    assert np.array_equal(Yd, Yh)
    assert _rel(Yh, C.to_dense() @ X) <= 1e-13


def test_batch_ragged_leaves_and_limits():
    w = I.plain_1d(1000)
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    X = np.random.default_rng(5).standard_normal((w.n, 4096))
    Y = A.matvec_batch(X)
    assert _rel(Y[:, :50], A.to_dense() @ X[:, :50]) <= 1e-13
    with pytest.raises(h2.H2Error):
        A.matvec_batch(np.zeros((w.n, 4097)))
