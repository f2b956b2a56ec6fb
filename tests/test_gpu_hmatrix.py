"""H-matrix output variant (h2_mul_h): the product after accumulation and
agglomeration, before the nested-basis recompression (Section 5.1; the
standard H-matrix approximation the paper's product passes through).

Parity: the oracle's factors of every admissible target block (MulResult.
factors, before recompression) and its dense inadmissible blocks, expanded
densely, against the GPU's expansion, block by block (1e-10); the
agglomeration bound eps/3 per block against the exact product."""
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


def oracle_hmatrix_dense(res):
    C = res.C
    D = C.dense()  # inadmissible leaves as in the H^2 result
    for b in O.block_leaves(C.blocks):
        if b.adm:
            L, R = res.factors[id(b)]
            D[np.ix_(b.t.idx, b.s.idx)] = L @ R.T
    return D


CASES = [(I.grid_2d(32), 1e-6), (I.grid_2d(64), 1e-6), (I.plain_1d(1000), 1e-4),
         (I.sphere_3d(2048), 1e-6)]


@pytest.mark.parametrize("w,eps", CASES, ids=[f"{w.name}-{e:g}" for w, e in CASES])
def test_hmatrix_product_matches_oracle(w, eps):
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
    Ch = h2.mul_h(A, B, eps)
    X, Y = build_pair(w)
    res = O.multiply(X, Y, eps)
    Do = oracle_hmatrix_dense(res)
    Dg = Ch.to_dense()
    Z = X.dense() @ Y.dense()
    worst_o = worst_z = 0.0
    ranks_o = []
    for b in O.block_leaves(res.C.blocks):
        ix = np.ix_(b.t.idx, b.s.idx)
        nz = np.linalg.norm(Z[ix], 2) or 1.0
        worst_o = max(worst_o, np.linalg.norm(Dg[ix] - Do[ix], 2) / nz)
        worst_z = max(worst_z, np.linalg.norm(Dg[ix] - Z[ix], 2) / nz)
        if b.adm:
            ranks_o.append(res.factors[id(b)][0].shape[1])
    assert worst_o <= 1e-10, worst_o
    assert worst_z <= eps / 3 * (1 + 1e-6), worst_z
    # agglomerated blocks carry the oracle's truncated ranks; accumulated ones 2k
    assert sorted(Ch.ranks().tolist()) == sorted(ranks_o)


def test_hmatrix_errors_and_free():
    w = I.plain_1d(256)
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    C = h2.mul_h(A, A, 1e-6)
    assert C.device_bytes() > 0
    C.free()
    C.free()  # idempotent in the binding
    with pytest.raises(h2.H2Error):
        h2.mul_h(A, A, -1.0)
