"""Small seeded cases shared by the oracle pins and the GPU parity tests."""
import numpy as np

from oracle import h2oracle as O
from paper_2403_01566_gb300 import inputs as I


def build_pair(w, tree=None):
    X = O.build_h2(w.points, w.kernel_a.kind, w.kernel_a.kparam(), w.eta, w.leaf_size, w.order, tree=tree)
    Y = O.build_h2(w.points, w.kernel_b.kind, w.kernel_b.kparam(), w.eta, w.leaf_size, w.order, tree=X.rows)
    return X, Y


def small_workloads():
    """Small cases spanning 1D/2D/3D, several levels and ragged leaves."""
    return [
        I.plain_1d(256),
        I.plain_1d(1000),                            # ragged: leaves of 31 and 32 points
        I.grid_2d(32),                               # 1024 grid points, k = 16
        I.square_2d(1500, seed=7, leaf=32, order=3),  # ragged 2D, k = 9
        I.cube_3d(1200, seed=11, leaf=40, order=2),   # 3D, k = 8
    ]


def block_rel_errors(C, Z):
    return [(e / z if z > 0 else e, adm) for e, z, adm, _ in O.blockwise_errors(C, Z)]
