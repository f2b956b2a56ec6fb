"""Chained products with variable-rank inputs: the product C is itself an
H^2-matrix input (adaptive ranks, stored padded with zero columns), and is
squared again (G -> G^2 -> G^4).  The GPU chain is compared with the oracle's
chain (each oracle product takes the oracle's previous result) block by block
(1e-10, as for single products), and every product meets the per-block bound
against the dense product of its own operands.
"""
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


def _worst(Cg, Co, Z, blocks):
    wo = wz = 0.0
    for b in O.block_leaves(blocks):
        ix = np.ix_(b.t.idx, b.s.idx)
        nz = np.linalg.norm(Z[ix], 2) or 1.0
        wo = max(wo, np.linalg.norm(Cg[ix] - Co[ix], 2) / nz)
        wz = max(wz, np.linalg.norm(Cg[ix] - Z[ix], 2) / nz)
    return wo, wz


@pytest.mark.parametrize("w,eps", [(I.grid_2d(32), 1e-6), (I.plain_1d(1024), 1e-8)], ids=lambda v: getattr(v, "name", str(v)))
def test_repeated_squaring_matches_oracle_chain(w, eps):
    A, B = (h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order),
            h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order))
    X, Y = build_pair(w)
    G = h2.mul(A, B, eps)
    Go = O.multiply(X, Y, eps).C
    for step in range(2):  # G^2, then G^4
        Gg_dense = G.to_dense()
        H = h2.mul(G, G, eps)
        res = O.multiply(Go, Go, eps)
        Zo = Go.dense() @ Go.dense()
        d_oracle, _ = _worst(H.to_dense(), res.C.dense(), Zo, res.C.blocks)
        _, d_exact = _worst(H.to_dense(), res.C.dense(), Gg_dense @ Gg_dense, res.C.blocks)
        assert d_oracle <= 1e-10, (step, d_oracle)
        assert d_exact <= eps, (step, d_exact)
        rr, rc = H.ranks()
        assert list(rr) == [res.ranks_row[c.id] for c in O.all_clusters(Go.rows)]
        assert list(rc) == [res.ranks_col[c.id] for c in O.all_clusters(Go.cols)]
        G, Go = H, res.C
