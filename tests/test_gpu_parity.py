"""GPU parity: the CUDA product against the CPU oracle (element by element on
small cases, by sampled columns and invariants at the full 128 x 128 grid
size), plus the edge cases of the boundary.

Tolerances: the FP64 path must agree with the oracle's dense-expanded product
within 1e-10 block-relative (both compute the same algorithm in FP64; the
difference is rounding, amplified at most by the gaps of the truncated
singular values), reproduce A*B to 1e-12 at eps = 0, and satisfy the
block-relative bound eps against the exact product.
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


def gpu_pair(w):
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
    return A, B


def blockrel(Cg, Co, Zref, C_oracle_blocks):
    worst_o = worst_z = 0.0
    for b in O.block_leaves(C_oracle_blocks):
        ix = np.ix_(b.t.idx, b.s.idx)
        nz = np.linalg.norm(Zref[ix], 2) or 1.0
        worst_o = max(worst_o, np.linalg.norm(Cg[ix] - Co[ix], 2) / nz)
        worst_z = max(worst_z, np.linalg.norm(Cg[ix] - Zref[ix], 2) / nz)
    return worst_o, worst_z


CASES = [
    (I.plain_1d(1024), 1e-6),
    (I.plain_1d(1000), 1e-4),                    # ragged leaves (31/32 points)
    (I.grid_2d(32), 1e-6),
    (I.grid_2d(64), 1e-6),                       # several tiles and agglomeration depths
    (I.square_2d(1500, seed=7, leaf=32, order=3), 1e-6),
    (I.cube_3d(1200, seed=11, leaf=40, order=2), 1e-4),
    # k = 64 (3D, order 4): factor widths 2k = 128, merges 256 wide
    (I.sphere_3d(2048), 1e-6),
    (I.sphere_3d(2048), 1e-4),
    (I.cube_3d(2048, seed=13, leaf=64, order=4), 1e-6),
]


@pytest.mark.parametrize("w,eps", CASES, ids=[f"{w.name}-{e:g}" for w, e in CASES])
def test_product_matches_oracle(w, eps):
    A, B = gpu_pair(w)
    C = h2.mul(A, B, eps)
    Cg = C.to_dense()
    X, Y = build_pair(w)
    res = O.multiply(X, Y, eps)
    Z = X.dense() @ Y.dense()
    d_oracle, d_exact = blockrel(Cg, res.C.dense(), Z, res.C.blocks)
    assert d_oracle <= 1e-10, d_oracle
    assert d_exact <= eps, d_exact
    rr, rc = C.ranks()
    assert list(rr) == [res.ranks_row[c.id] for c in O.all_clusters(X.rows)]
    assert list(rc) == [res.ranks_col[c.id] for c in O.all_clusters(Y.cols)]
    st = C.info()
    assert st.nagglomerated == res.agglomerated


@pytest.mark.parametrize("w", [I.plain_1d(256), I.plain_1d(500), I.grid_2d(16)], ids=lambda w: w.name)
def test_exact_product_eps0(w):
    A, B = gpu_pair(w)
    C = h2.mul(A, B, 0.0, max_rank=64)
    X, Y = build_pair(w)
    Z = X.dense() @ Y.dense()
    Cg = C.to_dense()
    worst = 0.0
    for b in O.block_leaves(O.build_block_tree(X.rows, Y.cols, w.eta)):
        ix = np.ix_(b.t.idx, b.s.idx)
        worst = max(worst, np.linalg.norm(Cg[ix] - Z[ix], 2) / (np.linalg.norm(Z[ix], 2) or 1.0))
    assert worst <= 1e-12, worst


def test_inputs_match_oracle_build():
    """h2_build gives the same H^2 matrix (same trees, blocks and values to rounding)."""
    w = I.grid_2d(32)
    A, _ = gpu_pair(w)
    X, _ = build_pair(w)
    assert np.array_equal(A.permutation(), X.rows.idx)
    Ad, Xd = A.to_dense(), X.dense()
    assert np.max(np.abs(Ad - Xd)) <= 1e-13 * np.max(np.abs(Xd))
    st = A.info()
    leaves = O.block_leaves(X.blocks)
    assert st.nadm == sum(b.adm for b in leaves) and st.ninadm == sum(not b.adm for b in leaves)


def test_matvec_against_dense():
    w = I.plain_1d(1024)
    A, _ = gpu_pair(w)
    X, _ = build_pair(w)
    x = I.random_vector(w.n, 5)
    y = A.matvec(x)
    ref = X.dense() @ x
    assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
    xt = torch.tensor(x, device="cuda")
    yt = A.matvec(xt).cpu().numpy()
    assert np.array_equal(yt, y)


def test_product_is_deterministic():
    w = I.grid_2d(32)
    A, B = gpu_pair(w)
    C1 = h2.mul(A, B, 1e-6).to_dense()
    C2 = h2.mul(A, B, 1e-6).to_dense()
    assert np.array_equal(C1, C2)


def test_errors():
    w = I.plain_1d(256)
    A, B = gpu_pair(w)
    with pytest.raises(h2.H2Error) as e:
        h2.mul(A, B, -1.0)
    assert e.value.code == h2.H2_EINVAL
    other = h2.build(I.plain_1d(256, seed_offset=1).points, w.kernel_a, w.eta, w.leaf_size, w.order)
    with pytest.raises(h2.H2Error) as e:
        h2.mul(A, other, 1e-6)
    assert e.value.code == h2.H2_ETREE
    with pytest.raises(h2.H2Error) as e:
        h2.mul(A, B, 0.0, max_rank=2)      # exact product needs higher ranks
    assert e.value.code == h2.H2_ERANK


def test_degenerate_single_leaf():
    """n <= leaf size: the root is a leaf, C is one dense block."""
    w = I.plain_1d(20)
    A, B = gpu_pair(w)
    C = h2.mul(A, B, 1e-6)
    X, Y = build_pair(w)
    assert np.allclose(C.to_dense(), X.dense() @ Y.dense(), rtol=0, atol=1e-13 * np.abs(X.dense()).max() ** 2 * 20)


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_full_size_grid_against_oracle(eps):
    """128 x 128 grid, A = -log|x-y|/(2 pi), B = exp(-|x-y|^2/0.1) at the
    three tolerances of the workload (eps = 1e-6 is the benchmark's):
    identical ranks, and C x equal to the oracle's C x within 1e-10 for
    random x; C x against A (B x) within the bound."""
    w = I.grid_2d(128, eps)
    A, B = gpu_pair(w)
    # eps = 1e-8 needs ranks up to 44 (the oracle's), above the default cap of
    # 32 for k = 16: the product refuses (H2_ERANK) rather than truncate
    if eps < 1e-7:
        with pytest.raises(h2.H2Error) as ei:
            h2.mul(A, B, w.eps)
        assert ei.value.code == h2.H2_ERANK
    C = h2.mul(A, B, w.eps, max_rank=64 if eps < 1e-7 else 0)
    X, Y = build_pair(w)
    res = O.multiply(X, Y, w.eps)
    rr, rc = C.ranks()
    assert list(rr) == [res.ranks_row[c.id] for c in O.all_clusters(X.rows)]
    assert list(rc) == [res.ranks_col[c.id] for c in O.all_clusters(Y.cols)]
    for seed in (1, 2, 3):
        x = I.random_vector(w.n, seed)
        yg = C.matvec(x)
        yo = res.C.matvec(x)
        assert np.linalg.norm(yg - yo) <= 1e-10 * np.linalg.norm(yo)
        yab = X.matvec(Y.matvec(x))
        assert np.linalg.norm(yg - yab) <= eps * np.sqrt(2 * 32) * np.linalg.norm(yab)


def test_plan_shared_by_operands_of_the_same_structure():
    """A cached plan serves every operand pair of the same structure: it holds
    no numeric data.  A second left factor with another kernel (same points,
    same trees, same block tree) reuses the plan of the first product and must
    still reproduce its own oracle product."""
    w = I.grid_2d(32)
    A1, B = gpu_pair(w)
    C1 = h2.mul(A1, B, 1e-6)
    k2 = I.KernelSpec(I.KERNEL_EXP, 2.0, 0.5, 0.3)
    A2 = h2.build(w.points, k2, w.eta, w.leaf_size, w.order)
    C2 = h2.mul(A2, B, 1e-6)
    X2 = O.build_h2(w.points, k2.kind, k2.kparam(), w.eta, w.leaf_size, w.order)
    Y = O.build_h2(w.points, w.kernel_b.kind, w.kernel_b.kparam(), w.eta, w.leaf_size, w.order, tree=X2.rows)
    res = O.multiply(X2, Y, 1e-6)
    Z = X2.dense() @ Y.dense()
    d_oracle, d_exact = blockrel(C2.to_dense(), res.C.dense(), Z, res.C.blocks)
    assert d_oracle <= 1e-10, d_oracle
    assert d_exact <= 1e-6, d_exact
    # and the first product is untouched by the second
    X1, Y1 = build_pair(w)
    res1 = O.multiply(X1, Y1, 1e-6)
    d1, _ = blockrel(C1.to_dense(), res1.C.dense(), X1.dense() @ Y1.dense(), res1.C.blocks)
    assert d1 <= 1e-10, d1


@pytest.mark.parametrize("m", [32, 64])
def test_grid_eps_1e8_with_rank_cap_64(m):
    """eps = 1e-8 (the tightest tolerance of the 2D grid workload) with
    max_rank = 64: same result and ranks as the oracle."""
    w = I.grid_2d(m)
    A, B = gpu_pair(w)
    C = h2.mul(A, B, 1e-8, max_rank=64)
    X, Y = build_pair(w)
    res = O.multiply(X, Y, 1e-8)
    Z = X.dense() @ Y.dense()
    d_oracle, d_exact = blockrel(C.to_dense(), res.C.dense(), Z, res.C.blocks)
    assert d_oracle <= 1e-10, d_oracle
    assert d_exact <= 1e-8, d_exact
    rr, rc = C.ranks()
    assert list(rr) == [res.ranks_row[c.id] for c in O.all_clusters(X.rows)]
