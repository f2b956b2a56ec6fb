"""Plain CPU FP64 oracle of adaptive H^2-matrix multiplication with
block-relative error control (S. Boerm, "Adaptive multiplication of
H^2-matrices with block-relative error control", arXiv 2403.01566).

TEST INFRASTRUCTURE ONLY.  This module is the independent checker of the CUDA
library: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path; both take
their inputs from ``paper_2403_01566_gb300.inputs``.

It follows the paper step by step, in numpy float64, with recursive data
structures and no blocking or reordering beyond what the paper states:

* cluster trees (Def. 1), block trees (Def. 2, eq. (4)), admissibility (eq. (2));
* H^2-matrices by tensor Chebyshev interpolation (eq. (3), transfer matrices
  from the identity theorem, Def. 3 / eq. (5), Def. 4);
* basis products P_{XY,s} = W_{X,s}^* V_{Y,s} (Section 4.1);
* basis trees with yield, mul, finish, add, split, uniform, nearfield
  (Defs. 8-9, Section 4.2) and the product added to a basis tree (Section 4.3);
* accumulators with the four cases and splitting (Def. 5, Sections 3.2-3.3,
  basis-tree form of the split in Section 4.3);
* coarsening by agglomeration with the row-then-column error control
  (Section 5.1 and its Remark);
* H^2 recompression with row*/col* sets, condensed blocks, weighted
  block-relative error control, projection climb and coupling matrices
  (Sections 5.2-5.3).

Readings of points where the paper is silent:

* R1  ``eta`` here is the factor in  max(diam) <= eta * dist  (eq. (2) with
      2*eta_paper = eta).
* R2  Omega_t is the tight axis-parallel bounding box of the cluster's points;
      diam is its diagonal, dist the Euclidean box distance.
* R3  Clusters are split by cardinality-balanced bisection along the longest
      box edge (stable sort by that coordinate, first child gets floor(|t|/2)
      points); every cluster above the depth D = min{d : ceil(n/2^d) <= leaf}
      is split, so all leaves lie on level D.
* R4  First-kind Chebyshev points per axis, x fastest in the tensor index;
      box axes narrower than 1e-6 * (root diagonal) are widened to that width
      for interpolation only.
* R5  Nystroem matrices g(x_i, x_j) with a prescribed diagonal value.
* R8  The target block tree of C is the admissibility block tree of (T_I, T_K)
      with the same eta; an admissible target leaf whose induced structure is
      finer is agglomerated.
* R9  A semi-uniform block A W^* + V B^* is factored as [A, V] [W, B]^*; a block
      carrying a dense nearfield part (leaf level only) is factored as (G, I).
* R10 Truncation keeps the singular values sigma_j > tol (tol relative to
      sigma_1 for agglomeration, absolute on the weighted panels for the
      bases); eps = 0 keeps every singular value.
* R11 theta = 1/4 (sigma = 2 children), weighted tolerance
      eps_side * sqrt(1 - 2 theta).
* R12 eps_hat is split into eps_hat/3 for agglomeration (further divided by
      2mn) and eps_hat/4 for each of the row and the column basis, so that
      every admissible block of C satisfies ||C_b - (AB)_b|| <= eps_hat ||(AB)_b||.
* R13 Block norms ||G^c_b||_2 are computed exactly (a lower bound of the
      spectral norm as the paper allows, with equality).
* R-agg The admissible target block's induced sub-blocks, refined to the
      deepest level of its induced subtree, form the n x m block matrix of the
      coarsening Remark; rows are agglomerated first (left to right), then the
      rows (top to bottom), with eps = eps_c / (2 m n).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Work counters of the method (measurement only; they change no arithmetic).
# Every dense operation of the product is counted where it happens:
#   gemm  a @ b of an (m x k) by a (k x n) matrix: 2 m n k flops
#   qr    Householder QR of an m x n matrix, R only: 2 n^2 (m - n/3) for
#         m >= n (2 m^2 (n - m/3) otherwise); forming the thin Q doubles it
#   svd   thin SVD by the R-SVD operation counts of Golub and Van Loan
#         (Matrix Computations, Section 8.6): singular values only
#         2 m n^2 + 2 n^3, with the thin U 6 m n^2 + 11 n^3, with U and V
#         6 m n^2 + 20 n^3 (m >= n, n <= m by transposition)
#   norm  spectral norm = the largest singular value (svd count, values only)
# Bytes: each operation reads its operands and writes its result once
# (8 bytes per double).  Elementwise sums and scalings (O(k^2) per node
# against the O(k^3) of the products) are not counted.
# --------------------------------------------------------------------------
class Work:
    KINDS = ("gemm", "qr", "svd", "norm")

    def __init__(self):
        self.reset()

    def reset(self):
        self.flops = {k: 0.0 for k in self.KINDS}
        self.bytes = {k: 0.0 for k in self.KINDS}
        self.calls = {k: 0 for k in self.KINDS}

    def add(self, kind, flops, nbytes):
        self.flops[kind] += flops
        self.bytes[kind] += nbytes
        self.calls[kind] += 1

    def snapshot(self):
        return {"flops": dict(self.flops), "bytes": dict(self.bytes), "calls": dict(self.calls)}


WORK = Work()


def _shape2(a):
    return (a.shape[0], 1) if a.ndim == 1 else a.shape


def mm(a, b):
    """a @ b, counted as a GEMM."""
    out = a @ b
    m, k = _shape2(a)
    n = 1 if b.ndim == 1 else b.shape[1]
    WORK.add("gemm", 2.0 * m * n * k, 8.0 * (a.size + b.size + out.size))
    return out


def _qr_flops(m, n):
    return 2.0 * n * n * (m - n / 3.0) if m >= n else 2.0 * m * m * (n - m / 3.0)


def qr_r(a):
    """R factor of the thin QR of a (counted without forming Q)."""
    _, r = np.linalg.qr(a)
    m, n = a.shape
    WORK.add("qr", _qr_flops(m, n), 8.0 * (a.size + r.size))
    return r


def qr_full(a):
    """Thin QR a = Q R, counted with the formation of Q."""
    q, r = np.linalg.qr(a)
    m, n = a.shape
    WORK.add("qr", 2.0 * _qr_flops(m, n), 8.0 * (a.size + q.size + r.size))
    return q, r


def _svd_flops(m, n, vectors):
    if m < n:
        m, n = n, m
    if vectors == 0:
        return 2.0 * m * n * n + 2.0 * n ** 3
    if vectors == 1:
        return 6.0 * m * n * n + 11.0 * n ** 3
    return 6.0 * m * n * n + 20.0 * n ** 3


def svd_u(a):
    """Thin SVD: U, sigma (right singular vectors not used)."""
    u, sig, _ = np.linalg.svd(a, full_matrices=False)
    WORK.add("svd", _svd_flops(a.shape[0], a.shape[1], 1), 8.0 * (a.size + u.size + sig.size))
    return u, sig


def svd_uv(a):
    """Thin SVD: U, sigma, V^*."""
    u, sig, vh = np.linalg.svd(a, full_matrices=False)
    WORK.add("svd", _svd_flops(a.shape[0], a.shape[1], 2), 8.0 * (a.size + u.size + sig.size + vh.size))
    return u, sig, vh


def block_norm(g):
    """Spectral norm ||g||_2 of a condensed block (Section 5.3; computed
    exactly, reading R13)."""
    if min(g.shape) == 0:
        return 0.0
    WORK.add("norm", _svd_flops(g.shape[0], g.shape[1], 0), 8.0 * g.size)
    return float(np.linalg.norm(g, 2))


def basis_weight(theta, level_s, level_t, nrm):
    """Weight omega_sr = theta^((level(s) - level(t)) / 2) ||G^c_tr||_2 of a block
    (t, r) seen at a descendant s of t (Section 5.3)."""
    return theta ** ((level_s - level_t) / 2.0) * nrm

# --------------------------------------------------------------------------
# Kernel functions (R5/R6)
# --------------------------------------------------------------------------
KERNEL_LOG, KERNEL_INV, KERNEL_GAUSS, KERNEL_EXP = 0, 1, 2, 3


def kernel_eval(kind, kparam, x, y):
    """g(x, y) for arrays of points x (a, d), y (b, d) -> (a, b); no diagonal rule."""
    scale, _, width, _ = kparam
    diff = x[:, None, :] - y[None, :, :]
    r2 = np.sum(diff * diff, axis=2)
    with np.errstate(divide="ignore", invalid="ignore"):
        if kind == KERNEL_LOG:
            return -scale * 0.5 * np.log(r2)
        if kind == KERNEL_INV:
            return scale / np.sqrt(r2)
        if kind == KERNEL_GAUSS:
            return scale * np.exp(-r2 / width)
        if kind == KERNEL_EXP:
            return scale * np.exp(-np.sqrt(r2) / width)
    raise ValueError("unknown kernel")


def kernel_block(kind, kparam, points, rows, cols):
    """Nystroem block g(x_i, x_j) for original indices rows x cols, with the
    diagonal value for i == j (R5)."""
    g = kernel_eval(kind, kparam, points[rows], points[cols])
    eq = rows[:, None] == cols[None, :]
    if np.any(eq):
        g = np.where(eq, kparam[1], g)
    return g


# --------------------------------------------------------------------------
# Cluster tree (Def. 1) with the readings R2/R3
# --------------------------------------------------------------------------
class Cluster:
    __slots__ = ("idx", "level", "lo", "hi", "children", "parent", "id", "off")

    def __init__(self, idx, level, lo, hi):
        self.idx = idx            # original point indices, in cluster order
        self.level = level
        self.lo = lo
        self.hi = hi
        self.children = []
        self.parent = None
        self.id = -1
        self.off = 0              # offset of the first index in the permuted order

    @property
    def size(self):
        return len(self.idx)

    @property
    def is_leaf(self):
        return not self.children


def _bbox(points, idx):
    p = points[idx]
    return p.min(axis=0), p.max(axis=0)


def tree_depth(n, leaf_size):
    d = 0
    while -(-n // (1 << d)) > leaf_size:
        d += 1
    return d


def build_cluster_tree(points, leaf_size):
    """Balanced bisection (R3).  Returns the root; clusters get ids in
    level order (breadth first, children in order)."""
    n, dim = points.shape
    depth = tree_depth(n, leaf_size)

    def rec(idx, level):
        lo, hi = _bbox(points, idx)
        c = Cluster(idx, level, lo, hi)
        if level < depth:
            ext = [float(hi[a]) - float(lo[a]) for a in range(dim)]
            axis = 0
            for a in range(1, dim):
                if ext[a] > ext[axis]:
                    axis = a
            order = np.argsort(points[idx, axis], kind="stable")
            sidx = idx[order]
            h = len(idx) // 2
            for part in (sidx[:h], sidx[h:]):
                ch = rec(part, level + 1)
                ch.parent = c
                c.children.append(ch)
            c.idx = np.concatenate([ch.idx for ch in c.children])
        return c

    root = rec(np.arange(n), 0)
    # ids in breadth-first order and offsets
    queue, cid = [root], 0
    while queue:
        nxt = []
        for c in queue:
            c.id = cid
            cid += 1
            nxt.extend(c.children)
        queue = nxt

    def set_off(c, off):
        c.off = off
        o = off
        for ch in c.children:
            set_off(ch, o)
            o += ch.size

    set_off(root, 0)
    return root


def all_clusters(root):
    out, queue = [], [root]
    while queue:
        out.extend(queue)
        queue = [ch for c in queue for ch in c.children]
    return out


def leaves_of(c):
    if c.is_leaf:
        return [c]
    return [lf for ch in c.children for lf in leaves_of(ch)]


def descendants_at(c, level):
    if c.level == level:
        return [c]
    return [d for ch in c.children for d in descendants_at(ch, level)]


def diam(c):
    acc = 0.0
    for a in range(len(c.lo)):
        g = float(c.hi[a]) - float(c.lo[a])
        acc += g * g
    return math.sqrt(acc)


def dist(t, s):
    acc = 0.0
    for a in range(len(t.lo)):
        g = max(0.0, float(s.lo[a]) - float(t.hi[a]), float(t.lo[a]) - float(s.hi[a]))
        acc += g * g
    return math.sqrt(acc)


def admissible(t, s, eta):
    """eq. (2) with the factor eta = 2*eta_paper (R1)."""
    return max(diam(t), diam(s)) <= eta * dist(t, s)


# --------------------------------------------------------------------------
# Block tree (Def. 2, eq. (4), recursive construction of Section 2)
# --------------------------------------------------------------------------
class Block:
    __slots__ = ("t", "s", "adm", "children", "parent")

    def __init__(self, t, s, adm, parent=None):
        self.t, self.s, self.adm = t, s, adm
        self.children = []
        self.parent = parent

    @property
    def is_leaf(self):
        return not self.children


def block_children_pairs(t, s):
    """eq. (4)."""
    if t.is_leaf:
        return [(t, sc) for sc in s.children]
    if s.is_leaf:
        return [(tc, s) for tc in t.children]
    return [(tc, sc) for tc in t.children for sc in s.children]


def build_block_tree(t, s, eta, parent=None):
    if admissible(t, s, eta):
        return Block(t, s, True, parent)
    b = Block(t, s, False, parent)
    if not (t.is_leaf and s.is_leaf):
        b.children = [build_block_tree(tc, sc, eta, b) for tc, sc in block_children_pairs(t, s)]
    return b


def block_leaves(b):
    if b.is_leaf:
        return [b]
    return [lf for c in b.children for lf in block_leaves(c)]


def all_blocks(b):
    out = [b]
    for c in b.children:
        out.extend(all_blocks(c))
    return out


# --------------------------------------------------------------------------
# Chebyshev interpolation (eq. (3), transfer matrices of Section 2)
# --------------------------------------------------------------------------
def cheb_nodes(lo, hi, m):
    nu = np.arange(m)
    return 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos((2 * nu + 1) * math.pi / (2 * m))


def lagrange_1d(nodes, x):
    """L[j](x) for all nodes j and points x -> (len(x), m)."""
    m = len(nodes)
    out = np.ones((len(x), m))
    for j in range(m):
        for i in range(m):
            if i != j:
                out[:, j] *= (x - nodes[i]) / (nodes[j] - nodes[i])
    return out


class Interp:
    """Per-cluster interpolation boxes and points (R4)."""

    def __init__(self, root, order):
        self.m = order
        self.dim = len(root.lo)
        self.k = order ** self.dim
        rootdiag = diam(root)
        self.minw = 1e-6 * rootdiag if rootdiag > 0 else 1e-6
        self.nodes = {}
        for c in all_clusters(root):
            axes = []
            for a in range(self.dim):
                lo, hi = float(c.lo[a]), float(c.hi[a])
                if hi - lo < self.minw:
                    mid = 0.5 * (lo + hi)
                    lo, hi = mid - 0.5 * self.minw, mid + 0.5 * self.minw
                axes.append(cheb_nodes(lo, hi, order))
            self.nodes[c.id] = axes

    def lagrange(self, c, pts):
        """ell_{c,nu}(pts) -> (len(pts), k), tensor index with x fastest."""
        out = np.ones((len(pts), 1))
        for a in range(self.dim):
            la = lagrange_1d(self.nodes[c.id][a], pts[:, a])
            # new index = nu_prev + m^a * nu_a  (x fastest)
            out = (la[:, :, None] * out[:, None, :]).reshape(len(pts), -1)
        return out

    def points(self, c):
        """Tensor interpolation points xi_{c,nu} -> (k, dim), x fastest."""
        axes = self.nodes[c.id]
        grids = np.meshgrid(*axes[::-1], indexing="ij")
        return np.stack([g.ravel() for g in grids[::-1]], axis=1)


# --------------------------------------------------------------------------
# Cluster bases and H^2-matrices (Defs. 3-4)
# --------------------------------------------------------------------------
class Basis:
    """Cluster basis: leaf matrices and transfer matrices E_{t'} (eq. (5))."""

    def __init__(self, root, leaf, trans, rank):
        self.root = root
        self.leaf = leaf      # id -> |t| x k_t for leaves
        self.trans = trans    # id -> k_t' x k_parent for non-root clusters
        self.rank = rank      # id -> k_t
        self._full = {}

    def full(self, c):
        """V_t reconstructed through the transfer matrices."""
        if c.id in self._full:
            return self._full[c.id]
        if c.is_leaf:
            v = self.leaf[c.id]
        else:
            v = np.vstack([mm(self.full(ch), self.trans[ch.id]) for ch in c.children])
        self._full[c.id] = v
        return v


class H2:
    def __init__(self, rows, cols, blocks, V, W, S, N, points=None):
        self.rows, self.cols, self.blocks = rows, cols, blocks
        self.V, self.W = V, W      # row basis (T_I), column basis (T_J)
        self.S = S                 # id(block) -> coupling
        self.N = N                 # id(block) -> dense nearfield
        self.points = points

    def dense_block(self, b):
        """G|_{t x s} for a block b of the block tree (cluster order)."""
        if b.is_leaf:
            if b.adm:
                return mm(mm(self.V.full(b.t), self.S[id(b)]), self.W.full(b.s).T)
            return self.N[id(b)]
        out = np.zeros((b.t.size, b.s.size))
        for c in b.children:
            ro, co = c.t.off - b.t.off, c.s.off - b.s.off
            out[ro:ro + c.t.size, co:co + c.s.size] = self.dense_block(c)
        return out

    def dense(self):
        """Dense matrix in the original index order."""
        d = self.dense_block(self.blocks)
        out = np.empty_like(d)
        out[np.ix_(self.rows.idx, self.cols.idx)] = d
        return out

    def matvec(self, x):
        """y = G x in O(nk): forward transform, coupling, backward transform,
        nearfield (standard H^2 matrix-vector multiplication, Section 2)."""
        xp = x[self.cols.idx]
        xhat = {}

        def fwd(s):
            if s.is_leaf:
                xhat[s.id] = self.W.leaf[s.id].T @ xp[s.off:s.off + s.size]
            else:
                acc = np.zeros(self.W.rank[s.id])
                for ch in s.children:
                    fwd(ch)
                    acc += self.W.trans[ch.id].T @ xhat[ch.id]
                xhat[s.id] = acc
        fwd(self.cols)
        yhat = {c.id: np.zeros(self.V.rank[c.id]) for c in all_clusters(self.rows)}
        yp = np.zeros(self.rows.size)
        for b in block_leaves(self.blocks):
            if b.adm:
                yhat[b.t.id] += self.S[id(b)] @ xhat[b.s.id]
            else:
                yp[b.t.off:b.t.off + b.t.size] += self.N[id(b)] @ xp[b.s.off:b.s.off + b.s.size]

        def bwd(t, carry):
            v = yhat[t.id] + carry
            if t.is_leaf:
                yp[t.off:t.off + t.size] += self.V.leaf[t.id] @ v
            else:
                for ch in t.children:
                    bwd(ch, self.V.trans[ch.id] @ v)
        bwd(self.rows, np.zeros(self.V.rank[self.rows.id]))
        y = np.empty_like(yp)
        y[self.rows.idx] = yp
        return y


    # ---- restricted products, for checking blocks of a product at sizes
    # where the product itself is out of the oracle's reach ----------------
    def _leaves_by_col(self):
        if not hasattr(self, "_bycol"):
            self._bycol = {}
            for b in block_leaves(self.blocks):
                self._bycol.setdefault(b.s.id, []).append(b)
        return self._bycol

    def _leaves_by_row(self):
        if not hasattr(self, "_byrow"):
            self._byrow = {}
            for b in block_leaves(self.blocks):
                self._byrow.setdefault(b.t.id, []).append(b)
        return self._byrow

    def matmat_cluster(self, c, Xc):
        """Y = G|_{I x c} Xc for a column cluster c and Xc (|c| x m), rows in
        the row tree's cluster order: the matrix-vector product of Section 2
        on columns supported in c.  The forward transform runs over c's
        subtree and up its ancestors (the other clusters see zero), then the
        couplings of the admissible leaves whose column cluster is among
        them, the backward transform and the nearfield leaves inside c."""
        m = Xc.shape[1]
        xhat = {}

        def fwd(s):
            lo = s.off - c.off
            if s.is_leaf:
                xhat[s.id] = self.W.leaf[s.id].T @ Xc[lo:lo + s.size]
            else:
                acc = np.zeros((self.W.rank[s.id], m))
                for ch in s.children:
                    fwd(ch)
                    acc += self.W.trans[ch.id].T @ xhat[ch.id]
                xhat[s.id] = acc
        fwd(c)
        a = c
        while a.parent is not None:
            xhat[a.parent.id] = self.W.trans[a.id].T @ xhat[a.id]
            a = a.parent
        bycol = self._leaves_by_col()
        yhat = {}
        Y = np.zeros((self.rows.size, m))
        for sid, xs in xhat.items():
            for b in bycol.get(sid, []):
                if b.adm:
                    v = self.S[id(b)] @ xs
                    yhat[b.t.id] = yhat[b.t.id] + v if b.t.id in yhat else v
                else:
                    lo = b.s.off - c.off
                    Y[b.t.off:b.t.off + b.t.size] += self.N[id(b)] @ Xc[lo:lo + b.s.size]

        def bwd(t, carry):
            v = yhat.get(t.id)
            if carry is not None:
                v = carry if v is None else v + carry
            if t.is_leaf:
                if v is not None:
                    Y[t.off:t.off + t.size] += self.V.leaf[t.id] @ v
            else:
                for ch in t.children:
                    bwd(ch, None if v is None else self.V.trans[ch.id] @ v)
        bwd(self.rows, None)
        return Y

    def rows_matmat(self, t, Z):
        """(G Z)|_t for a row cluster t and Z (n_cols x m) in the column tree's
        cluster order: the forward transform of Z over the whole column tree,
        the couplings of the admissible leaves whose row cluster is t, one of
        its ancestors or descendants, the backward transform restricted to t
        and the nearfield leaves of rows inside t."""
        m = Z.shape[1]
        xhat = {}

        def fwd(s):
            if s.is_leaf:
                xhat[s.id] = self.W.leaf[s.id].T @ Z[s.off:s.off + s.size]
            else:
                acc = np.zeros((self.W.rank[s.id], m))
                for ch in s.children:
                    fwd(ch)
                    acc += self.W.trans[ch.id].T @ xhat[ch.id]
                xhat[s.id] = acc
        fwd(self.cols)
        byrow = self._leaves_by_row()
        out = np.zeros((t.size, m))
        # couplings of t's ancestors, pushed down to t through the transfers
        chain = []
        a = t
        while a is not None:
            chain.append(a)
            a = a.parent
        carry = None
        for a in reversed(chain):          # root first
            if carry is not None and a is not chain[-1]:
                carry = self.V.trans[a.id] @ carry
            for b in byrow.get(a.id, []):
                if b.adm:
                    v = self.S[id(b)] @ xhat[b.s.id]
                    carry = v if carry is None else carry + v
                elif a is t:
                    out += self.N[id(b)] @ Z[b.s.off:b.s.off + b.s.size]

        # t's own subtree: its couplings, pushed down with the ancestors' part
        def bwd(u, cu):
            v = cu
            if u is not t:
                for b in byrow.get(u.id, []):
                    if b.adm:
                        w = self.S[id(b)] @ xhat[b.s.id]
                        v = w if v is None else v + w
            if u.is_leaf:
                lo = u.off - t.off
                if v is not None:
                    out[lo:lo + u.size] += self.V.leaf[u.id] @ v
                if u is not t:
                    for b in byrow.get(u.id, []):
                        if not b.adm:
                            out[lo:lo + u.size] += self.N[id(b)] @ Z[b.s.off:b.s.off + b.s.size]
            else:
                for ch in u.children:
                    bwd(ch, None if v is None else self.V.trans[ch.id] @ v)
        bwd(t, carry)
        return out


def product_block(X, Y, t, r):
    """(X Y)|_{t x r} (cluster order) of two H^2-matrices sharing the middle
    cluster tree, through their matrix-vector products: Y on the unit
    vectors of r (Y|_{J x r}), then the rows t of X applied to it."""
    return X.rows_matmat(t, Y.matmat_cluster(r, np.eye(r.size)))


def chebyshev_basis(root, interp, points):
    leaf, trans, rank = {}, {}, {}
    for c in all_clusters(root):
        rank[c.id] = interp.k
        if c.is_leaf:
            leaf[c.id] = interp.lagrange(c, points[c.idx])
        for ch in c.children:
            # E_{t'}(nu', nu) = ell_{t,nu}(xi_{t',nu'})
            trans[ch.id] = interp.lagrange(c, interp.points(ch))
    return Basis(root, leaf, trans, rank)


def build_h2(points, kind, kparam, eta, leaf_size, order, tree=None):
    """H^2 approximation of the Nystroem matrix by tensor Chebyshev
    interpolation (eq. (3)): leaf V_t(i,nu) = ell_{t,nu}(x_i), transfer
    E_{t'}(nu',nu) = ell_{t,nu}(xi_{t',nu'}), coupling S_ts = g(xi_t, xi_s),
    dense nearfield g(x_i, x_j)."""
    points = np.asarray(points, dtype=np.float64)
    root = tree if tree is not None else build_cluster_tree(points, leaf_size)
    interp = Interp(root, order)
    basis = chebyshev_basis(root, interp, points)
    bt = build_block_tree(root, root, eta)
    S, N = {}, {}
    for b in block_leaves(bt):
        if b.adm:
            S[id(b)] = kernel_eval(kind, kparam, interp.points(b.t), interp.points(b.s))
        else:
            N[id(b)] = kernel_block(kind, kparam, points, b.t.idx, b.s.idx)
    h = H2(root, root, bt, basis, basis, S, N, points)
    h.eta = eta
    h.kernel = (kind, tuple(kparam))
    return h


# --------------------------------------------------------------------------
# Basis products (Section 4.1): P_{XY,s} = W_{X,s}^* V_{Y,s}
# --------------------------------------------------------------------------
def basis_products(WX, VY, root):
    """Leaves directly, inner clusters through the transfer matrices:
    P_s = sum_{s'} F_{X,s'}^* P_{s'} E_{Y,s'}."""
    P = {}

    def rec(s):
        if s.is_leaf:
            P[s.id] = mm(WX.leaf[s.id].T, VY.leaf[s.id])
        else:
            acc = np.zeros((WX.rank[s.id], VY.rank[s.id]))
            for ch in s.children:
                rec(ch)
                acc += mm(mm(WX.trans[ch.id].T, P[ch.id]), VY.trans[ch.id])
            P[s.id] = acc
    rec(root)
    return P


# --------------------------------------------------------------------------
# Basis trees (Defs. 8-9, Section 4.2); copy-on-write, never mutated
# --------------------------------------------------------------------------
def _mm(a, b):
    """Matrix product with None standing for the identity."""
    if a is None:
        return b
    if b is None:
        return a
    return mm(a, b)


class BT:
    """Basis tree node.  Leaf cluster: (C, N, M); inner: (C, M) or
    (C, M, kids).  M = None stands for the identity."""
    __slots__ = ("t", "C", "M", "N", "kids")

    def __init__(self, t, C, M=None, N=None, kids=None):
        self.t, self.C, self.M, self.N, self.kids = t, C, M, N, kids

    def ncols(self):
        return self.C.shape[1] if self.M is None else self.M.shape[1]


def bt_zero(t, krow, kcol):
    if t.is_leaf:
        return BT(t, np.zeros((krow, kcol)), None, np.zeros((t.size, kcol)))
    return BT(t, np.zeros((krow, kcol)))


def bt_yield(a, basis):
    """Def. 9."""
    t = a.t
    if t.is_leaf:
        return _mm(mm(basis.full(t), a.C) + a.N, a.M)
    if a.kids is None:
        return _mm(mm(basis.full(t), a.C), a.M)
    rows = [mm(basis.full(tc), mm(basis.trans[tc.id], a.C)) + bt_yield(ac, basis)
            for tc, ac in zip(t.children, a.kids)]
    return _mm(np.vstack(rows), a.M)


def bt_mul(a, X):
    """mul(alpha, X): yield(mul(alpha, X)) = yield(alpha) X."""
    if X is None:
        return a
    return BT(a.t, a.C, _mm(a.M, X), a.N, a.kids)


def bt_finish(a):
    """finish(alpha): apply the pending transformation."""
    if a.M is None:
        return a
    if a.t.is_leaf:
        return BT(a.t, mm(a.C, a.M), None, mm(a.N, a.M))
    if a.kids is None:
        return BT(a.t, mm(a.C, a.M))
    return BT(a.t, mm(a.C, a.M), None, None, [bt_mul(c, a.M) for c in a.kids])


def bt_split(a, basis):
    """split(alpha) for alpha = (C, M) on a non-leaf cluster."""
    t = a.t
    CM = _mm(a.C, a.M)
    kids = []
    for tc in t.children:
        c = mm(basis.trans[tc.id], CM)
        kids.append(BT(tc, c, None, np.zeros((tc.size, c.shape[1]))) if tc.is_leaf else BT(tc, c))
    return BT(t, np.zeros((a.C.shape[0], CM.shape[1])), None, None, kids)


def bt_add(a, b, basis):
    """add(alpha, beta): yield(add) = yield(alpha) + yield(beta)."""
    t = a.t
    if t.is_leaf:
        return BT(t, _mm(a.C, a.M) + _mm(b.C, b.M), None, _mm(a.N, a.M) + _mm(b.N, b.M))
    if a.kids is None and b.kids is None:
        return BT(t, _mm(a.C, a.M) + _mm(b.C, b.M))
    if a.kids is None:
        a = bt_split(a, basis)
    if b.kids is None:
        b = bt_split(b, basis)
    C = _mm(a.C, a.M) + _mm(b.C, b.M)
    kids = [bt_add(bt_mul(ai, a.M), bt_mul(bi, b.M), basis) for ai, bi in zip(a.kids, b.kids)]
    return BT(t, C, None, None, kids)


def bt_uniform(t, C):
    """uniform(C) (eq. (11)): yield = V_{X,t} C."""
    if t.is_leaf:
        return BT(t, C, None, np.zeros((t.size, C.shape[1])))
    return BT(t, C)


def bt_nearfield(t, Z, krow):
    """nearfield(Z) (eq. (10)): yield = Z, t a leaf."""
    return BT(t, np.zeros((krow, Z.shape[1])), None, Z)


def bt_restrict(a, tc, basis):
    """Restriction of yield(alpha) to the rows of a child tc (Section 4.3)."""
    CM = _mm(a.C, a.M)
    push = mm(basis.trans[tc.id], CM)
    if a.kids is None:
        if tc.is_leaf:
            return BT(tc, push, None, np.zeros((tc.size, push.shape[1])))
        return BT(tc, push)
    i = a.t.children.index(tc)
    ai = bt_finish(bt_mul(a.kids[i], a.M))
    return BT(tc, ai.C + push, None, ai.N, ai.kids)


# --------------------------------------------------------------------------
# The two sides of the product.  Side A builds A_tr = X|_{t x s} V_{Y,s} S
# (basis V_X, transfers E_X); side B builds B_tr = Y|_{s x r}^* W_{X,s} S
# (basis W_Y, transfers F_Y), i.e. the same algorithm on the adjoint.
# --------------------------------------------------------------------------
class Side:
    def __init__(self, left, right_basis_leaf, P, is_adjoint):
        self.left = left                   # H2 whose block tree is walked
        self.adj = is_adjoint
        self.basis = left.W if is_adjoint else left.V   # basis of the tree's rows
        self.descend_basis = right_basis_leaf           # basis over T_J (V_Y or W_X)
        self.P = P

    def row(self, b):
        return b.s if self.adj else b.t

    def col(self, b):
        return b.t if self.adj else b.s

    def coupling(self, b):
        S = self.left.S[id(b)]
        return S.T if self.adj else S

    def Pmat(self, s):
        return self.P[s.id].T if self.adj else self.P[s.id]

    def near(self, b):
        Nb = self.left.N[id(b)]
        return Nb.T if self.adj else Nb

    def children(self, b):
        # children of the (possibly adjoint) block, as (row, col, block)
        return [(self.row(c), self.col(c), c) for c in b.children]


def product_pieces(side, b, S):
    """The basis trees whose yields sum to Z|_{t x s} U_s S (Section 4.3): the
    block subtree of b walked level by level, the right factor carried down by
    U_{s'} = U_s E_{s'} (eq. (5)), so a child block (t', s') gets E_{s'} S when
    its column cluster is a child of s (S unchanged when s is a leaf).  Every
    leaf block contributes at its row cluster t': an admissible leaf the basis
    tree uniform(S_{t's'} P_{s'} S) of eq. (11), an inadmissible leaf
    nearfield(N_{t's'} U_{s'} S) of eq. (10).  Returns [(t', beta)]."""
    pieces = []
    level = [(b, S)]
    while level:
        deeper = []
        for blk, Sb in level:
            t, s = side.row(blk), side.col(blk)
            if blk.is_leaf:
                if blk.adm:
                    pieces.append((t, bt_uniform(t, mm(mm(side.coupling(blk), side.Pmat(s)), Sb))))
                else:
                    Z = mm(side.near(blk), mm(side.descend_basis.full(s), Sb))
                    pieces.append((t, bt_nearfield(t, Z, side.basis.rank[t.id])))
                continue
            for _, sc, c in side.children(blk):
                deeper.append((c, Sb if sc is s else mm(side.descend_basis.trans[sc.id], Sb)))
        level = deeper
    return pieces


def deposit(a, tgt, beta, basis):
    """yield(alpha) + yield(beta) restricted to the rows of tgt, tgt = alpha's
    cluster or a descendant: add(alpha, beta) at tgt (Section 4.2), reached
    through finish and split on the way down (both keep the yield)."""
    if a.t is tgt:
        return bt_add(a, beta, basis)
    a = bt_finish(a)
    if a.kids is None:
        a = bt_split(a, basis)
    i = next(j for j, tc in enumerate(a.t.children) if tc.off <= tgt.off < tc.off + tc.size)
    kids = list(a.kids)
    kids[i] = deposit(kids[i], tgt, beta, basis)
    return BT(a.t, a.C, None, None, kids)


def addproduct(side, b, S, a):
    """The basis tree alpha' with yield(alpha') = yield(alpha) + Z|_{t x s} U_s S,
    Z the side's matrix (X or Y^*) and U its partner basis (V_Y or W_X)
    (Section 4.3): the pieces of the product, each added at its row cluster."""
    for tgt, beta in product_pieces(side, b, S):
        a = deposit(a, tgt, beta, side.basis)
    return a


# --------------------------------------------------------------------------
# Accumulators (Def. 5, Sections 3.2-3.3 and 4.3)
# --------------------------------------------------------------------------
@dataclass
class Acc:
    t: Cluster
    r: Cluster
    alpha: BT
    beta: BT
    N: np.ndarray | None = None
    P: list = field(default_factory=list)   # pairs (X block (t,s), Y block (s,r))


class Product:
    """State of one product X*Y (the paper's Z = XY)."""

    def __init__(self, X, Y):
        self.X, self.Y = X, Y
        self.P = basis_products(X.W, Y.V, X.cols)
        self.sideA = Side(X, Y.V, self.P, False)
        self.sideB = Side(Y, X.W, self.P, True)
        self.kA = Y.W.rank        # column rank of A_tr lives on T_K (k of W_Y)
        self.kB = X.V.rank

    def new_acc(self, t, r):
        ka = self.Y.W.rank[r.id]
        kb = self.X.V.rank[t.id]
        return Acc(t, r, bt_zero(t, self.X.V.rank[t.id], ka), bt_zero(r, self.Y.W.rank[r.id], kb))

    def add(self, acc, xb, yb):
        """The four cases of Section 3.2 (case 1 first when both apply, R17)."""
        if yb.is_leaf and yb.adm:                       # case 1
            acc.alpha = addproduct(self.sideA, xb, self.Y.S[id(yb)], acc.alpha)
        elif xb.is_leaf and xb.adm:                     # case 2
            acc.beta = addproduct(self.sideB, yb, self.X.S[id(xb)].T, acc.beta)
        elif xb.is_leaf or yb.is_leaf:                  # case 3
            prod = mm(self.X.dense_block(xb), self.Y.dense_block(yb))
            acc.N = prod if acc.N is None else acc.N + prod
        else:                                           # case 4
            acc.P.append((xb, yb))

    def split(self, acc, pairs):
        """Split accumulator (t,r) into its children (t',r'); pairs lists the
        children in order."""
        out = []
        for tc, rc in pairs:
            alpha = acc.alpha if tc is acc.t else bt_restrict(acc.alpha, tc, self.X.V)
            if rc is not acc.r:
                alpha = bt_mul(alpha, self.Y.W.trans[rc.id].T)
            beta = acc.beta if rc is acc.r else bt_restrict(acc.beta, rc, self.Y.W)
            if tc is not acc.t:
                beta = bt_mul(beta, self.X.V.trans[tc.id].T)
            N = None
            if acc.N is not None:
                ro, co = tc.off - acc.t.off, rc.off - acc.r.off
                N = acc.N[ro:ro + tc.size, co:co + rc.size]
            child = Acc(tc, rc, alpha, beta, N)
            for xb, yb in acc.P:
                for xc in xb.children:
                    if xc.t is not tc:
                        continue
                    for yc in yb.children:
                        if yc.t is xc.s and yc.s is rc:
                            self.add(child, xc, yc)
            out.append(child)
        return out

    def factor(self, acc):
        """Low-rank factorization of accu(A_tr) with P = {} (R9)."""
        assert not acc.P
        A = bt_yield(acc.alpha, self.X.V)
        B = bt_yield(acc.beta, self.Y.W)
        L = np.hstack([A, self.X.V.full(acc.t)])
        R = np.hstack([self.Y.W.full(acc.r), B])
        if acc.N is not None:
            return (mm(L, R.T) + acc.N, np.eye(acc.r.size))
        return (L, R)

    def dense(self, acc):
        L, R = self.factor(acc)
        return mm(L, R.T)


def split_pairs(t, r):
    return block_children_pairs(t, r)


# --------------------------------------------------------------------------
# Coarsening (Section 5.1) with its error-control Remark
# --------------------------------------------------------------------------
def _truncate(sig, tol_rel, eps_is_zero):
    if eps_is_zero:
        return len(sig)
    if len(sig) == 0 or sig[0] == 0.0:
        return 0
    return int(np.sum(sig > tol_rel * sig[0]))


def merge_columns(f1, f2, eps, eps_is_zero):
    """Agglomerate [L1 R1^*, L2 R2^*] (same rows): QR of the block-diagonal
    right factor, condensed matrix, SVD, truncation."""
    (L1, R1), (L2, R2) = f1, f2
    Q1, r1 = qr_full(R1)
    Q2, r2 = qr_full(R2)
    G = np.hstack([mm(L1, r1.T), mm(L2, r2.T)])
    U, sig, Vh = svd_uv(G)
    k = _truncate(sig, eps, eps_is_zero)
    Vk = Vh[:k].T
    Qv = np.vstack([mm(Q1, Vk[:Q1.shape[1]]), mm(Q2, Vk[Q1.shape[1]:])])
    return (U[:, :k] * sig[:k], Qv)


def merge_rows(f1, f2, eps, eps_is_zero):
    """Agglomerate [L1 R1^*; L2 R2^*] (same columns): QR of [R1 R2],
    condensed [L1 r_1^*; L2 r_2^*], SVD, truncation (Section 5.1)."""
    (L1, R1), (L2, R2) = f1, f2
    Q, r = qr_full(np.hstack([R1, R2]))
    m1 = R1.shape[1]
    G = np.vstack([mm(L1, r[:, :m1].T), mm(L2, r[:, m1:].T)])
    U, sig, Vh = svd_uv(G)
    k = _truncate(sig, eps, eps_is_zero)
    return (U[:, :k] * sig[:k], mm(Q, Vh[:k].T))


# --------------------------------------------------------------------------
# The whole product (Sections 3-5)
# --------------------------------------------------------------------------
@dataclass
class MulResult:
    C: H2
    factors: dict          # id(target adm leaf) -> (L, R) before recompression
    ranks_row: dict
    ranks_col: dict
    norms: dict
    agglomerated: int
    stats: dict


def multiply(X, Y, eps, theta=0.25):
    """Approximate Z = X*Y by an H^2-matrix with adaptive isometric bases and
    block-relative error eps in every admissible block (R8-R13)."""
    assert X.cols is Y.rows or X.cols.idx.tolist() == Y.rows.idx.tolist()
    eps_is_zero = eps == 0.0
    eps_c = eps / 3.0
    eps_side = eps / 4.0
    WORK.reset()
    prod = Product(X, Y)
    tI, tK = X.rows, Y.cols
    target = build_block_tree(tI, tK, X.eta)
    factors, dense_out = {}, {}
    stats = {"agglomerated": 0, "terminal": 0}

    def induced(acc, depth, out):
        """Split while P is not empty; collect terminal accumulators."""
        if not acc.P:
            out.append((acc, depth))
            return
        assert not (acc.t.is_leaf and acc.r.is_leaf)
        for ch in prod.split(acc, split_pairs(acc.t, acc.r)):
            induced(ch, depth + 1, out)

    def refine(acc, depth, d):
        if depth == d:
            return [acc]
        out = []
        for ch in prod.split(acc, split_pairs(acc.t, acc.r)):
            out.extend(refine(ch, depth + 1, d))
        return out

    def agglomerate(acc):
        terms = []
        induced(acc, 0, terms)
        d = max(dp for _, dp in terms)
        cells = []
        for a, dp in terms:
            cells.extend(refine(a, dp, d))
        rows = descendants_at(acc.t, acc.t.level + d)
        cols = descendants_at(acc.r, acc.r.level + d)
        grid = {(a.t.id, a.r.id): prod.factor(a) for a in cells}
        n, m = len(rows), len(cols)
        e = eps_c / (2.0 * m * n)
        row_f = []
        for ti in rows:
            f = grid[(ti.id, cols[0].id)]
            for rj in cols[1:]:
                f = merge_columns(f, grid[(ti.id, rj.id)], e, eps_is_zero)
            row_f.append(f)
        f = row_f[0]
        for g in row_f[1:]:
            f = merge_rows(f, g, e, eps_is_zero)
        return f

    def process(acc, tb):
        if tb.children:
            kids = prod.split(acc, [(c.t, c.s) for c in tb.children])
            for ka, kb in zip(kids, tb.children):
                process(ka, kb)
        elif tb.adm:
            stats["terminal"] += 1
            if acc.P:
                stats["agglomerated"] += 1
                factors[id(tb)] = agglomerate(acc)
            else:
                factors[id(tb)] = prod.factor(acc)
        else:
            assert not acc.P
            dense_out[id(tb)] = prod.dense(acc)

    root = prod.new_acc(tI, tK)
    prod.add(root, X.blocks, Y.blocks)
    process(root, target)

    # ---------------- H^2 recompression (Sections 5.2-5.3) ----------------
    adm = [b for b in block_leaves(target) if b.adm]
    tol = eps_side * math.sqrt(1.0 - 2.0 * theta)
    Gc, Gcc, norms = {}, {}, {}
    for b in adm:
        L, R = factors[id(b)]
        Rr = qr_r(R)                       # B_tr = Q_tr R_tr
        Gc[id(b)] = mm(L, Rr.T)            # condensed G^c_tr
        Rl = qr_r(L)                       # adjoint: A_tr = Q' R'
        Gcc[id(b)] = mm(R, Rl.T)
        norms[id(b)] = block_norm(Gc[id(b)])

    def build_basis(root, blocks_of, cond, cluster_of):
        """Weighted adaptive cluster basis (Sections 5.2-5.3), bottom-up."""
        rows_star = {}

        def star(c, inherited):
            own = blocks_of.get(c.id, [])
            rows_star[c.id] = inherited + own
            for ch in c.children:
                star(ch, rows_star[c.id])
        star(root, [])
        leaf, trans, rank = {}, {}, {}
        ghat = {}                       # (cluster id, id(b)) -> V_t^* G^c_b|_t

        def rec(c):
            for ch in c.children:
                rec(ch)
            cols, keys = [], []
            for b in rows_star[c.id]:
                nb = norms[id(b)]
                if nb == 0.0:
                    continue
                tb = cluster_of(b)
                w = basis_weight(theta, c.level, tb.level, nb)
                if c.is_leaf:
                    ro = c.off - tb.off
                    blk = cond[id(b)][ro:ro + c.size]
                else:
                    blk = np.vstack([ghat[(ch.id, id(b))] for ch in c.children])
                cols.append(blk / w)
                keys.append((b, blk))
            nrows = c.size if c.is_leaf else sum(rank[ch.id] for ch in c.children)
            if cols:
                G = np.hstack(cols)
                U, sig = svd_u(G)
                k = len(sig) if eps_is_zero else int(np.sum(sig > tol))
                Vh = U[:, :k]
            else:
                Vh = np.zeros((nrows, 0))
            rank[c.id] = Vh.shape[1]
            if c.is_leaf:
                leaf[c.id] = Vh
            else:
                o = 0
                for ch in c.children:
                    trans[ch.id] = Vh[o:o + rank[ch.id]]
                    o += rank[ch.id]
            for b, blk in keys:
                ghat[(c.id, id(b))] = mm(Vh.T, blk)
        rec(root)
        return Basis(root, leaf, trans, rank)

    row_blocks, col_blocks = {}, {}
    for b in adm:
        row_blocks.setdefault(b.t.id, []).append(b)
        col_blocks.setdefault(b.s.id, []).append(b)
    Vnew = build_basis(tI, row_blocks, Gc, lambda b: b.t)
    Wnew = build_basis(tK, col_blocks, Gcc, lambda b: b.s)

    S, N = {}, {}
    for b in adm:
        L, R = factors[id(b)]
        S[id(b)] = mm(mm(Vnew.full(b.t).T, L), mm(Wnew.full(b.s).T, R).T)
    for b in block_leaves(target):
        if not b.adm:
            N[id(b)] = dense_out[id(b)]
    C = H2(tI, tK, target, Vnew, Wnew, S, N)
    C.eta = X.eta
    stats["work"] = WORK.snapshot()
    return MulResult(C, factors, Vnew.rank, Wnew.rank, norms, stats["agglomerated"], stats)


# --------------------------------------------------------------------------
# Checks used by the tests (dense, brute force)
# --------------------------------------------------------------------------
def blockwise_errors(C, Zd):
    """For every leaf block b of C: (||C_b - Z_b||_2, ||Z_b||_2, adm, b),
    Zd the dense reference in the original index order."""
    Cd = C.dense()
    out = []
    for b in block_leaves(C.blocks):
        ri, ci = b.t.idx, b.s.idx
        zb = Zd[np.ix_(ri, ci)]
        cb = Cd[np.ix_(ri, ci)]
        out.append((np.linalg.norm(cb - zb, 2), np.linalg.norm(zb, 2), b.adm, b))
    return out
