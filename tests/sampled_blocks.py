"""Exact blocks (AB)|_{t x r} of a product at sizes where the oracle's own
product is out of reach, from the oracle's H^2-matrices and their restricted
matrix-vector products (oracle.h2oracle.product_block), computed in worker
processes started with `spawn` (they hold no CUDA state).

Used by the full-size GPU tests: the GPU's C_b is compared with these blocks
against the block-relative bound of Section 5.3."""
import numpy as np

from oracle import h2oracle as O
from paper_2403_01566_gb300 import inputs as I

_W = {}


def _sphere_pair(n):
    if n not in _W:
        w = I.sphere_3d(n)
        X = O.build_h2(w.points, w.kernel_a.kind, w.kernel_a.kparam(), w.eta, w.leaf_size, w.order)
        _W[n] = (w, X, {c.id: c for c in O.all_clusters(X.rows)})
    return _W[n]


def sphere_blocks(n, pairs):
    """(A A)|_{t x r} for the cluster-id pairs (t, r) of the n-point sphere
    workload, rows and columns in cluster order (t.idx, r.idx)."""
    _, X, cl = _sphere_pair(n)
    return [O.product_block(X, X, cl[t], cl[r]) for t, r in pairs]


def sample_admissible_blocks(X, eta, per_level, seed):
    """Seeded sample of the admissible leaves of the target block tree of
    X*X, per cluster level: {level: [(t_id, r_id), ...]}."""
    rng = np.random.default_rng(seed)
    target = O.build_block_tree(X.rows, X.cols, eta)
    by_level = {}
    for b in O.block_leaves(target):
        if b.adm:
            by_level.setdefault(b.t.level, []).append((b.t.id, b.s.id))
    out = {}
    for lvl, bl in sorted(by_level.items()):
        k = min(len(bl), per_level.get(lvl, 0))
        if k:
            idx = rng.choice(len(bl), size=k, replace=False)
            out[lvl] = [bl[i] for i in sorted(idx)]
    return out
