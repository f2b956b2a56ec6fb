"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: brute-force
dense linear algebra on tiny inputs, closed forms, invariants of the
definitions, or the error bounds the paper proves.  A planted mistake in the
oracle (last test) must be caught by these pins.
"""
import math

import numpy as np
import pytest

from oracle import h2oracle as O
from paper_2403_01566_gb300 import inputs as I
from tests.oracle_cases import block_rel_errors, build_pair, small_workloads

RNG = np.random.default_rng(1234)


# ---------------------------------------------------------------- trees ----
@pytest.mark.parametrize("n,leaf", [(1, 4), (5, 4), (256, 32), (1000, 32), (1000, 62), (777, 10)])
def test_cluster_tree_partition_and_balance(n, leaf):
    """Def. 1: children partition the parent; leaves partition I (Section 2);
    reading R3: all leaves on one level, |leaf| <= leaf size."""
    pts = I.uniform_points(n, 2, 99)
    root = O.build_cluster_tree(pts, leaf)
    assert sorted(root.idx.tolist()) == list(range(n))
    leaves = O.leaves_of(root)
    assert sorted(np.concatenate([lf.idx for lf in leaves]).tolist()) == list(range(n))
    depth = O.tree_depth(n, leaf)
    assert all(lf.level == depth and 1 <= lf.size <= leaf for lf in leaves)
    for c in O.all_clusters(root):
        if c.children:
            assert np.array_equal(np.concatenate([ch.idx for ch in c.children]), c.idx)
        p = pts[c.idx]
        assert np.array_equal(p.min(axis=0), c.lo) and np.array_equal(p.max(axis=0), c.hi)


def test_block_tree_partition_and_admissibility():
    """Def. 2: the leaves partition I x J; admissible leaves satisfy eq. (2);
    inadmissible leaves pair two leaf clusters (Section 2)."""
    pts = I.uniform_points(300, 2, 5)
    root = O.build_cluster_tree(pts, 16)
    bt = O.build_block_tree(root, root, 2.0)
    cover = np.zeros((300, 300), dtype=int)
    for b in O.block_leaves(bt):
        cover[np.ix_(b.t.idx, b.s.idx)] += 1
        if b.adm:
            assert max(O.diam(b.t), O.diam(b.s)) <= 2.0 * O.dist(b.t, b.s)
        else:
            assert b.t.is_leaf and b.s.is_leaf
    assert np.all(cover == 1)


def test_box_distance_closed_form():
    """R2: diam and dist of axis-parallel boxes."""
    a = O.Cluster(np.arange(1), 0, np.array([0.0, 0.0]), np.array([1.0, 2.0]))
    b = O.Cluster(np.arange(1), 0, np.array([4.0, 6.0]), np.array([5.0, 7.0]))
    assert O.diam(a) == pytest.approx(math.sqrt(5.0))
    assert O.dist(a, b) == pytest.approx(5.0)
    assert O.dist(a, a) == 0.0


# ------------------------------------------------------ interpolation ----
def test_chebyshev_nodes_closed_form():
    """R4: first-kind Chebyshev points (a+b)/2 + (b-a)/2 cos((2nu+1)pi/(2m))."""
    x = O.cheb_nodes(0.0, 1.0, 2)
    assert x[0] == pytest.approx(0.5 + 0.5 / math.sqrt(2.0))
    assert x[1] == pytest.approx(0.5 - 0.5 / math.sqrt(2.0))


def test_lagrange_is_cardinal_and_reproduces_polynomials():
    """eq. (3): ell_nu(xi_mu) = delta; interpolation of degree < m is exact."""
    nodes = O.cheb_nodes(-0.3, 1.7, 5)
    assert np.allclose(O.lagrange_1d(nodes, nodes), np.eye(5), atol=1e-14)
    x = np.linspace(-0.3, 1.7, 17)
    f = lambda z: 3 * z ** 4 - z ** 2 + 0.5
    approx = O.lagrange_1d(nodes, x) @ f(nodes)
    assert np.allclose(approx, f(x), rtol=0, atol=1e-12)


@pytest.mark.parametrize("w", [I.plain_1d(256), I.grid_2d(32), I.cube_3d(600, 3, leaf=40, order=3)],
                         ids=["1d", "2d", "3d"])
def test_nested_basis_identity(w):
    """eq. (5): V_t|_{t'} = V_{t'} E_{t'}, with V_t evaluated directly by the
    Lagrange polynomials of t (not through the transfer matrices)."""
    X, _ = build_pair(w)
    interp = O.Interp(X.rows, w.order)
    for c in O.all_clusters(X.rows):
        direct = interp.lagrange(c, w.points[c.idx])
        assert np.allclose(X.V.full(c), direct, rtol=0, atol=1e-11 * max(1.0, np.abs(direct).max()))


def test_h2_interpolation_converges_with_order():
    """eq. (3): the interpolation error of admissible blocks falls with the order."""
    pts = I.uniform_points(400, 2, 17)
    dense = O.kernel_block(0, (1.0, 1.0, 1.0, 0.0), pts, np.arange(400), np.arange(400))
    errs = []
    for order in (2, 4, 6):
        h = O.build_h2(pts, 0, (1.0, 1.0, 1.0, 0.0), 2.0, 32, order)
        errs.append(np.linalg.norm(h.dense() - dense) / np.linalg.norm(dense))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-4


def test_nearfield_and_diagonal_rule():
    """R5: inadmissible leaves hold g(x_i,x_j) exactly, with the diagonal value."""
    w = I.plain_1d(256)
    X, _ = build_pair(w)
    full = O.kernel_block(0, w.kernel_a.kparam(), w.points, np.arange(256), np.arange(256))
    d = X.dense()
    for b in O.block_leaves(X.blocks):
        if not b.adm:
            assert np.array_equal(d[np.ix_(b.t.idx, b.s.idx)], full[np.ix_(b.t.idx, b.s.idx)])
    assert np.all(np.diag(d) == 1.0)


def test_matvec_matches_dense():
    """Section 2: the O(nk) matrix-vector product equals the dense product."""
    w = I.grid_2d(32)
    X, _ = build_pair(w)
    x = RNG.standard_normal(w.n)
    assert np.allclose(X.matvec(x), X.dense() @ x, rtol=0, atol=1e-12 * np.abs(X.dense() @ x).max())


# ------------------------------------------------------ basis products ----
def test_basis_products_brute_force():
    """Section 4.1: P_{XY,s} = W_{X,s}^* V_{Y,s} for every cluster, against
    directly evaluated bases."""
    w = I.grid_2d(32)
    X, Y = build_pair(w)
    P = O.basis_products(X.W, Y.V, X.cols)
    interp = O.Interp(X.rows, w.order)
    for s in O.all_clusters(X.cols):
        Ws = interp.lagrange(s, w.points[s.idx])
        assert np.allclose(P[s.id], Ws.T @ Ws, rtol=0, atol=1e-11 * max(1, np.abs(P[s.id]).max()))


# ------------------------------------------------------ basis trees ----
def _random_tree(t, k, depth, rng):
    """Random basis tree over t with random pending transforms."""
    M = rng.standard_normal((k, k))
    C = rng.standard_normal((k, k))
    if t.is_leaf:
        return O.BT(t, C, M, rng.standard_normal((t.size, k)))
    if depth == 0:
        return O.BT(t, C, M)
    return O.BT(t, C, M, None, [_random_tree(c, k, depth - 1, rng) for c in t.children])


@pytest.fixture(scope="module")
def small_h2():
    return build_pair(I.plain_1d(256))


def test_basis_tree_operation_identities(small_h2):
    """Section 4.2: yield(mul(a,X)) = yield(a)X, yield(finish(a)) = yield(a),
    yield(split(a)) = yield(a), yield(add(a,b)) = yield(a)+yield(b); the yield
    itself checked against its definition (Def. 9) written densely."""
    X, _ = small_h2
    rng = np.random.default_rng(3)
    root = X.rows
    k = 4
    for depth in (0, 1, 3):
        a = _random_tree(root, k, depth, rng)
        b = _random_tree(root, k, 2, rng)
        Xm = rng.standard_normal((k, k))
        ya = O.bt_yield(a, X.V)
        assert np.allclose(O.bt_yield(O.bt_mul(a, Xm), X.V), ya @ Xm)
        assert np.allclose(O.bt_yield(O.bt_finish(a), X.V), ya)
        assert np.allclose(O.bt_yield(O.bt_add(a, b, X.V), X.V), ya + O.bt_yield(b, X.V))
    a = O.BT(root, rng.standard_normal((k, k)), rng.standard_normal((k, k)))
    assert np.allclose(O.bt_yield(O.bt_split(a, X.V), X.V), O.bt_yield(a, X.V))
    # Def. 9 for a two-level tree, written out densely
    t1, t2 = root.children
    a = _random_tree(root, k, 1, rng)
    rows = []
    for tc, ac in zip((t1, t2), a.kids):
        rows.append(X.V.full(tc) @ X.V.trans[tc.id] @ a.C + O.bt_yield(ac, X.V))
    assert np.allclose(O.bt_yield(a, X.V), np.vstack(rows) @ a.M)
    assert np.allclose(X.V.full(root), np.vstack([X.V.full(t1) @ X.V.trans[t1.id], X.V.full(t2) @ X.V.trans[t2.id]]))


def test_addproduct_matches_dense(small_h2):
    """Fig. 1: addproduct(X|_{t x s}, S, alpha) adds X|_{t x s} V_{Y,s} S."""
    X, Y = small_h2
    prod = O.Product(X, Y)
    rng = np.random.default_rng(5)
    for b in O.all_blocks(X.blocks)[:60]:
        S = rng.standard_normal((4, 4))
        a0 = _random_tree(b.t, 4, 2, rng)
        a1 = O.addproduct(prod.sideA, b, S, a0)
        ref = O.bt_yield(a0, X.V) + X.dense_block(b) @ Y.V.full(b.s) @ S
        assert np.allclose(O.bt_yield(a1, X.V), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_accumulator_cases_and_split_exact(small_h2):
    """Sections 3.2-3.3: each of the four cases adds exactly X|ts Y|sr, and
    splitting gives accu(A_{t'r'}) = accu(A_tr)|_{t' x r'}."""
    X, Y = small_h2
    prod = O.Product(X, Y)
    Z = X.dense() @ Y.dense()

    def accu(acc):
        M = O.bt_yield(acc.alpha, X.V) @ Y.W.full(acc.r).T + X.V.full(acc.t) @ O.bt_yield(acc.beta, Y.W).T
        if acc.N is not None:
            M = M + acc.N
        for xb, yb in acc.P:
            M = M + X.dense_block(xb) @ Y.dense_block(yb)
        return M

    cases = set()
    for xb in O.all_blocks(X.blocks):
        for yb in O.all_blocks(Y.blocks):
            if yb.t is not xb.s:
                continue
            acc = prod.new_acc(xb.t, yb.s)
            prod.add(acc, xb, yb)
            cases.add((bool(acc.P), acc.N is not None))
            ref = X.dense_block(xb) @ Y.dense_block(yb)
            assert np.allclose(accu(acc), ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    assert len(cases) >= 3
    root = prod.new_acc(X.rows, Y.cols)
    prod.add(root, X.blocks, Y.blocks)
    zp = Z[np.ix_(X.rows.idx, Y.cols.idx)]

    def walk(acc):
        got = accu(acc)
        ro, co = acc.t.off, acc.r.off
        ref = zp[ro:ro + acc.t.size, co:co + acc.r.size]
        assert np.allclose(got, ref, rtol=0, atol=1e-11 * np.abs(zp).max())
        if not acc.t.is_leaf:
            for ch in prod.split(acc, O.split_pairs(acc.t, acc.r)):
                walk(ch)
    walk(root)


# ------------------------------------------------------ coarsening ----
def test_agglomeration_merges_truncate_exactly():
    """Section 5.1: the merged factorization is the truncated SVD of the block
    matrix; its error is the largest dropped singular value <= eps*||G||."""
    rng = np.random.default_rng(8)
    L1, R1 = rng.standard_normal((30, 6)), rng.standard_normal((25, 6))
    L2, R2 = rng.standard_normal((30, 5)), rng.standard_normal((20, 5))
    G = np.hstack([L1 @ R1.T, L2 @ R2.T])
    sig = np.linalg.svd(G, compute_uv=False)
    for eps in (0.0, 1e-3, 0.2):
        L, R = O.merge_columns((L1, R1), (L2, R2), eps, eps == 0.0)
        k = L.shape[1]
        err = np.linalg.norm(G - L @ R.T, 2)
        dropped = sig[k] if k < len(sig) else 0.0
        assert err == pytest.approx(dropped, abs=1e-12 * sig[0])
        assert err <= eps * sig[0] + 1e-12 * sig[0]
    L3, R3 = rng.standard_normal((12, 4)), rng.standard_normal((25, 4))
    H = np.vstack([L1 @ R1.T, L3 @ R3.T])
    L, R = O.merge_rows((L1, R1), (L3, R3), 0.05, False)
    sH = np.linalg.svd(H, compute_uv=False)
    assert np.linalg.norm(H - L @ R.T, 2) <= 0.05 * sH[0] * (1 + 1e-12)


# ------------------------------------------------------ whole product ----
@pytest.mark.parametrize("w", small_workloads(), ids=lambda w: w.name)
def test_exact_product_at_eps0(w):
    """Sections 3-4: with eps = 0 (full ranks) C reproduces dense(A) dense(B)
    to rounding in every block (the exact product representation)."""
    X, Y = build_pair(w)
    res = O.multiply(X, Y, 0.0)
    Z = X.dense() @ Y.dense()
    errs = block_rel_errors(res.C, Z)
    assert max(e for e, _ in errs) < 1e-12


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
@pytest.mark.parametrize("w", small_workloads()[1:4], ids=lambda w: w.name)
def test_block_relative_bound(w, eps):
    """Section 5.3 with the coarsening Remark: every admissible block of C
    satisfies ||C_b - (AB)_b||_2 <= eps ||(AB)_b||_2; nearfield blocks are exact."""
    X, Y = build_pair(w)
    res = O.multiply(X, Y, eps)
    Z = X.dense() @ Y.dense()
    for e, adm in block_rel_errors(res.C, Z):
        assert e <= (eps if adm else 1e-12)


def test_output_bases_isometric():
    """Section 5.2: V_t^* V_t = I and W_r^* W_r = I for every cluster."""
    w = I.grid_2d(32, 1e-6)
    X, Y = build_pair(w)
    res = O.multiply(X, Y, 1e-6)
    for basis in (res.C.V, res.C.W):
        for c in O.all_clusters(res.C.rows):
            V = basis.full(c)
            assert np.allclose(V.T @ V, np.eye(V.shape[1]), rtol=0, atol=1e-13)


def test_agglomerated_blocks_within_coarsening_bound():
    """Coarsening Remark: agglomerated target blocks keep ||G - G~|| <= eps_c ||G||
    with eps_c = eps/3."""
    w = I.grid_2d(32, 1e-5)
    X, Y = build_pair(w)
    res = O.multiply(X, Y, 1e-5)
    assert res.agglomerated > 0
    Zp = (X.dense() @ Y.dense())
    for b in O.block_leaves(res.C.blocks):
        if b.adm:
            L, R = res.factors[id(b)]
            zb = Zp[np.ix_(b.t.idx, b.s.idx)]
            assert np.linalg.norm(L @ R.T - zb, 2) <= (1e-5 / 3) * np.linalg.norm(zb, 2) * (1 + 1e-9)


def test_identity_times_b_is_b():
    """Special case: A = I as an H^2 matrix (identity nearfield on diagonal
    leaves, zero couplings) gives C = B within eps in every block."""
    w = I.plain_1d(512, 1e-6)
    X, Y = build_pair(w)
    Id = O.H2(X.rows, X.cols, X.blocks, X.V, X.W,
              {k: np.zeros_like(v) for k, v in X.S.items()},
              {id(b): (np.eye(b.t.size) if b.t is b.s else np.zeros((b.t.size, b.s.size)))
               for b in O.block_leaves(X.blocks) if not b.adm})
    Id.eta = X.eta
    assert np.array_equal(Id.dense(), np.eye(w.n))
    res = O.multiply(Id, Y, 1e-6)
    for e, _ in block_rel_errors(res.C, Y.dense()):
        assert e <= 1e-6


def test_product_matvec_against_factors():
    """C x = A (B x) through the O(nk) matrix-vector products (eps = 0: to
    rounding; eps > 0: within the bound of the per-block errors)."""
    w = I.grid_2d(32)
    X, Y = build_pair(w)
    x = RNG.standard_normal(w.n)
    ref = X.matvec(Y.matvec(x))
    r0 = O.multiply(X, Y, 0.0)
    assert np.linalg.norm(r0.C.matvec(x) - ref) <= 1e-12 * np.linalg.norm(ref)
    r6 = O.multiply(X, Y, 1e-6)
    assert np.linalg.norm(r6.C.matvec(x) - ref) <= 1e-6 * math.sqrt(2 * 40) * np.linalg.norm(ref)


def test_planted_mistake_is_caught(monkeypatch):
    """A dropped transfer matrix in the basis-tree split must break the eps=0
    exactness pin."""
    w = I.plain_1d(256)
    X, Y = build_pair(w)

    def bad_split(a, basis):
        t = a.t
        CM = O._mm(a.C, a.M)
        kids = [O.BT(tc, CM.copy(), None, np.zeros((tc.size, CM.shape[1]))) if tc.is_leaf else O.BT(tc, CM.copy())
                for tc in t.children]
        return O.BT(t, np.zeros_like(CM), None, None, kids)

    monkeypatch.setattr(O, "bt_split", bad_split)
    res = O.multiply(X, Y, 0.0)
    Z = X.dense() @ Y.dense()
    assert max(e for e, _ in block_rel_errors(res.C, Z)) > 1e-6
