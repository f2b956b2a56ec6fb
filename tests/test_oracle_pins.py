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
    """Section 4.3: addproduct(X|_{t x s}, S, alpha) adds X|_{t x s} V_{Y,s} S."""
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


# ------------------------------------------------------ kernel functions ----
# Hand-computed values: ln 5 = 1.6094379124341003, ln 3 = 1.0986122886681098,
# ln 2 = 0.6931471805599453, e^-2.5 = 0.0820849986238988,
# e^-5 = 0.006737946999085467, e^-3 = 0.049787068367863944,
# 1/(2 pi) = 0.15915494309189535.
@pytest.mark.parametrize("spec,x,y,value", [
    (I.LOG, (0.0, 0.0), (3.0, 4.0), -1.6094379124341003),               # -log 5
    (I.LOG_2PI, (0.0, 0.0), (3.0, 4.0), -1.6094379124341003 * 0.15915494309189535),
    (I.LOG, (0.25,), (0.75,), 0.6931471805599453),                       # -log 0.5
    (I.LOG, (1.0, 2.0, 2.0), (0.0, 0.0, 0.0), -1.0986122886681098),     # -log 3
    (I.INV, (0.0, 0.0), (3.0, 4.0), 0.2),
    (I.INV, (1.0, 2.0, 2.0), (0.0, 0.0, 0.0), 1.0 / 3.0),
    (I.INV_4PI, (0.0, 0.0, 0.0), (0.0, 0.3, 0.4), 0.15915494309189535),  # 1/(4 pi 0.5)
    (I.GAUSS_01, (0.0, 0.0), (0.3, 0.4), 0.0820849986238988),            # exp(-0.25/0.1)
    (I.EXP, (0.0, 0.0), (3.0, 4.0), 0.006737946999085467),               # exp(-5)
    (I.EXP, (1.0, 2.0, 2.0), (0.0, 0.0, 0.0), 0.049787068367863944),    # exp(-3)
], ids=["log-r5", "log2pi-r5", "log-1d", "log-3d", "inv-r5", "inv-3d", "inv4pi", "gauss", "exp-r5", "exp-3d"])
def test_kernel_closed_forms(spec, x, y, value):
    """R5/R6: each kernel string of the workloads, evaluated at point pairs
    whose distance is known (the Pythagorean triples 3-4-5 and 1-2-2-3)."""
    g = O.kernel_eval(spec.kind, spec.kparam(), np.array([x]), np.array([y]))
    assert g.shape == (1, 1)
    assert g[0, 0] == pytest.approx(value, rel=1e-14, abs=0.0)
    # symmetric in its arguments
    assert O.kernel_eval(spec.kind, spec.kparam(), np.array([y]), np.array([x]))[0, 0] == g[0, 0]


@pytest.mark.parametrize("spec,diag", [(I.LOG, 1.0), (I.LOG_2PI, 1.0), (I.INV_4PI, 0.0), (I.INV, 0.0),
                                       (I.GAUSS_01, 1.0), (I.EXP, 1.0)])
def test_kernel_diagonal_rule(spec, diag):
    """R5: the Nystroem entry i == j takes the workload's diagonal value; off
    the diagonal the kernel is evaluated (here at distance 5 on a 3-4-5 pair)."""
    pts = np.array([[0.0, 0.0], [3.0, 4.0]])
    g = O.kernel_block(spec.kind, spec.kparam(), pts, np.arange(2), np.arange(2))
    assert g[0, 0] == diag and g[1, 1] == diag
    off = O.kernel_eval(spec.kind, spec.kparam(), pts[:1], pts[1:])[0, 0]
    assert g[0, 1] == off and g[1, 0] == off


# ------------------------------------------------ weighted recompression ----
THETA = 0.25


def _adm_blocks(res):
    return [b for b in O.block_leaves(res.C.blocks) if b.adm]


def _dense_factor(res, b):
    L, R = res.factors[id(b)]
    return L @ R.T


def _ancestors_or_self(c):
    out = []
    while c is not None:
        out.append(c)
        c = c.parent
    return out


def _basis_discrepancy(res, eps, row_side, leaves_only=False):
    """Sections 5.2-5.3, rebuilt by this test from the blocks before
    recompression and the oracle's output bases.  For every cluster t the
    weighted stacked matrix
        G_t = [ H_b / omega_{t,b} ]_b,   b = (t', r) admissible, t' = t or an
        ancestor of t,  omega = theta^((level t - level t')/2) ||G_b||_2,
    with H_b = G_b|_t for a leaf and H_b = [V_{t1}^* G_b|_{t1}; V_{t2}^* G_b|_{t2}]
    (the children's output bases) otherwise, must satisfy
        ||G_t - Vh_t Vh_t^* G_t||_2 = sigma_{k+1}(G_t)
    where Vh_t is the leaf basis V_t or the stacked transfer matrices
    [E_{t1}; E_{t2}] and k its rank, with the rank decision
    sigma_{k+1} <= tol < sigma_k, tol = (eps/4) sqrt(1 - 2 theta).  The blocks
    are used uncondensed: a right isometry changes neither singular values nor
    left singular vectors.  Returns the largest violation relative to sigma_1."""
    tol = (eps / 4.0) * math.sqrt(1.0 - 2.0 * THETA)
    basis = res.C.V if row_side else res.C.W
    root = res.C.rows if row_side else res.C.cols
    blocks_at, dense, nrm = {}, {}, {}
    for b in _adm_blocks(res):
        c = b.t if row_side else b.s
        blocks_at.setdefault(c.id, []).append(b)
        G = _dense_factor(res, b)
        dense[id(b)] = G if row_side else G.T
        nrm[id(b)] = np.linalg.svd(G, compute_uv=False)[0]
    worst = 0.0
    clusters = O.leaves_of(root) if leaves_only else O.all_clusters(root)
    for t in clusters:
        cols = []
        for anc in _ancestors_or_self(t):
            for b in blocks_at.get(anc.id, []):
                if nrm[id(b)] == 0.0:
                    continue
                G = dense[id(b)]
                w = THETA ** ((t.level - anc.level) / 2.0) * nrm[id(b)]
                if t.is_leaf:
                    ro = t.off - anc.off
                    H = G[ro:ro + t.size]
                else:
                    parts = []
                    for ch in t.children:
                        ro = ch.off - anc.off
                        parts.append(basis.full(ch).T @ G[ro:ro + ch.size])
                    H = np.vstack(parts)
                cols.append(H / w)
        if t.is_leaf:
            Vh = basis.leaf[t.id]
        else:
            Vh = np.vstack([basis.trans[ch.id] for ch in t.children])
        if not cols:
            assert Vh.shape[1] == 0
            continue
        Gt = np.hstack(cols)
        sig = np.linalg.svd(Gt, compute_uv=False)
        k = Vh.shape[1]
        dropped = sig[k] if k < len(sig) else 0.0
        err = np.linalg.norm(Gt - Vh @ (Vh.T @ Gt), 2)
        viol = abs(err - dropped) / sig[0]
        if dropped > tol * (1 + 1e-9):
            viol = max(viol, (dropped - tol) / sig[0])
        if k > 0 and sig[k - 1] <= tol * (1 - 1e-9):
            viol = max(viol, (tol - sig[k - 1]) / sig[0])
        worst = max(worst, viol)
    return worst


@pytest.fixture(scope="module")
def grid_products():
    out = {}
    for eps in (1e-4, 1e-6):
        w = I.grid_2d(32, eps)
        X, Y = build_pair(w)
        out[eps] = (X, Y, O.multiply(X, Y, eps))
    return out


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_weighted_blockwise_basis_bound(grid_products, eps):
    """Section 5.3: with the weights omega and tol = (eps/4) sqrt(1 - 2 theta),
    every admissible block b = (t, r) keeps
        ||G_b - V_t V_t^* G_b||_2 <= (eps/4) ||G_b||_2   (row basis)
        ||G_b - G_b W_r W_r^*||_2 <= (eps/4) ||G_b||_2   (column basis)
    with G_b the accumulated (or agglomerated) block before recompression."""
    _, _, res = grid_products[eps]
    worst_row = worst_col = 0.0
    for b in _adm_blocks(res):
        G = _dense_factor(res, b)
        nrm = np.linalg.svd(G, compute_uv=False)[0]
        V, W = res.C.V.full(b.t), res.C.W.full(b.s)
        er = np.linalg.norm(G - V @ (V.T @ G), 2) / nrm
        ec = np.linalg.norm(G - (G @ W) @ W.T, 2) / nrm
        assert er <= (eps / 4.0) * (1 + 1e-9)
        assert ec <= (eps / 4.0) * (1 + 1e-9)
        worst_row, worst_col = max(worst_row, er), max(worst_col, ec)
    # the bound is attained to within a small factor: the truncation is active
    assert worst_row > 0.02 * eps / 4.0 and worst_col > 0.02 * eps / 4.0


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
@pytest.mark.parametrize("row_side", [True, False], ids=["rows", "cols"])
def test_basis_error_is_largest_dropped_weighted_sigma(grid_products, eps, row_side):
    """Section 5.2: ||G_t - V_t V_t^* G_t||_2 = sigma_{k+1} for the weighted
    stacked matrix of every cluster (leaf bases and nested transfer matrices),
    with the rank chosen against tol (Section 5.3)."""
    _, _, res = grid_products[eps]
    # the equality holds to rounding (~1e-17 sigma_1); a planted weight
    # mistake misses it by 1e-12 sigma_1 or more (next test)
    assert _basis_discrepancy(res, eps, row_side) < 1e-13


def test_planted_weight_mistakes_are_caught(monkeypatch):
    """A wrong weight exponent sign, or the Frobenius norm in place of the
    spectral norm, must break the basis pin."""
    eps = 1e-2
    w = I.grid_2d(32, eps)
    X, Y = build_pair(w)
    assert _basis_discrepancy(O.multiply(X, Y, eps), eps, True) < 1e-13
    good = O.basis_weight
    monkeypatch.setattr(O, "basis_weight", lambda th, ls, lt, nrm: good(th, lt, ls, nrm))
    assert _basis_discrepancy(O.multiply(X, Y, eps), eps, True) > 1e-11
    monkeypatch.setattr(O, "basis_weight", good)
    monkeypatch.setattr(O, "block_norm", lambda g: float(np.linalg.norm(g)) if g.size else 0.0)
    assert _basis_discrepancy(O.multiply(X, Y, eps), eps, True) > 1e-11


# ------------------------------------------------------ work counters ----
def test_work_counters_count_the_operations():
    """The counters of the oracle: a GEMM of (m x k)(k x n) is 2mnk flops and
    reads/writes its three matrices; QR and SVD follow the stated formulas."""
    O.WORK.reset()
    a, b = np.ones((3, 5)), np.ones((5, 7))
    O.mm(a, b)
    assert O.WORK.flops["gemm"] == 2 * 3 * 5 * 7
    assert O.WORK.bytes["gemm"] == 8 * (15 + 35 + 21)
    O.qr_r(np.ones((10, 4)))
    assert O.WORK.flops["qr"] == pytest.approx(2 * 16 * (10 - 4 / 3))
    O.svd_u(np.ones((4, 10)))
    assert O.WORK.flops["svd"] == pytest.approx(6 * 10 * 16 + 11 * 64)


def test_work_grows_like_n_log_n():
    """Section 4 / Section 6: the work of a product grows like n k^2 log n at
    fixed k; doubling n on the 1D workload multiplies it by about
    2 (log 2n / log n), well below 4."""
    fl = []
    for n in (512, 1024, 2048):
        w = I.plain_1d(n, 1e-6)
        X, Y = build_pair(w)
        res = O.multiply(X, Y, w.eps)
        wk = res.stats["work"]
        fl.append(sum(wk["flops"].values()))
        assert wk["calls"]["gemm"] > 0 and wk["calls"]["qr"] > 0 and wk["calls"]["svd"] > 0
    assert 1.6 < fl[1] / fl[0] < 3.0 and 1.6 < fl[2] / fl[1] < 3.0


# ------------------------------------------- restricted matrix products ----
@pytest.mark.parametrize("w", [I.plain_1d(1000), I.grid_2d(32), I.cube_3d(1200, seed=11, leaf=40, order=2)],
                         ids=["1d", "2d", "3d"])
def test_restricted_products_match_dense(w):
    """The matrix-vector products restricted to one cluster (columns supported
    in c; rows of t) and the product blocks (XY)|_{t x r} built from them,
    against the dense matrices (cluster order), for every cluster and the
    first blocks of the block tree."""
    X, Y = build_pair(w)
    Xd, Yd = X.dense_block(X.blocks), Y.dense_block(Y.blocks)
    rng = np.random.default_rng(21)
    for c in O.all_clusters(X.rows):
        Xc = rng.standard_normal((c.size, 3))
        ref = Xd[:, c.off:c.off + c.size] @ Xc
        assert np.allclose(X.matmat_cluster(c, Xc), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        Z = rng.standard_normal((w.n, 2))
        ref2 = (Xd @ Z)[c.off:c.off + c.size]
        assert np.allclose(X.rows_matmat(c, Z), ref2, rtol=0, atol=1e-12 * np.abs(ref2).max())
    Zd = Xd @ Yd
    for b in O.all_blocks(X.blocks)[:80]:
        ref = Zd[b.t.off:b.t.off + b.t.size, b.s.off:b.s.off + b.s.size]
        got = O.product_block(X, Y, b.t, b.s)
        assert np.allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
