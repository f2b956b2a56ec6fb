"""Seeded synthetic inputs (point sets and workload descriptions).

This module holds no arithmetic of the multiplication method: it only draws
or places points and names the kernel functions and parameters of each
workload.  Both the CUDA path and the CPU oracle take their inputs from here.

The workloads stand in for the paper's boundary-element test matrices
(Section 6: single-layer operator on the unit sphere, double-layer operator on
the cube surface), which need meshes and quadrature that are not part of the
method.  Nystroem point matrices g(x_i, x_j) of the same kernel families on
seeded point sets replace them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20240303

# Kernel ids shared with the C ABI (h2_build_opts.kernel).
KERNEL_LOG = 0    # g(x,y) = -scale * log|x-y|
KERNEL_INV = 1    # g(x,y) = scale / |x-y|
KERNEL_GAUSS = 2  # g(x,y) = scale * exp(-|x-y|^2 / width)
KERNEL_EXP = 3    # g(x,y) = scale * exp(-|x-y| / width)


@dataclass(frozen=True)
class KernelSpec:
    """A kernel function id with its parameters.

    kparam = (scale, diagonal value, width, unused); the diagonal value is
    used for the entry i == j of the Nystroem matrix.
    """
    kind: int
    scale: float = 1.0
    diag: float = 0.0
    width: float = 1.0

    def kparam(self):
        return (float(self.scale), float(self.diag), float(self.width), 0.0)


LOG = KernelSpec(KERNEL_LOG, 1.0, 1.0)
LOG_2PI = KernelSpec(KERNEL_LOG, 1.0 / (2.0 * math.pi), 1.0)
GAUSS_01 = KernelSpec(KERNEL_GAUSS, 1.0, 1.0, 0.1)
INV_4PI = KernelSpec(KERNEL_INV, 1.0 / (4.0 * math.pi), 0.0)
INV = KernelSpec(KERNEL_INV, 1.0, 0.0)
EXP = KernelSpec(KERNEL_EXP, 1.0, 1.0, 1.0)


def uniform_points(n: int, dim: int, seed: int) -> np.ndarray:
    """n points uniform on [0,1]^dim, row-major (n, dim), float64."""
    rng = np.random.default_rng(seed)
    return rng.random((n, dim), dtype=np.float64)


def grid_points(m: int) -> np.ndarray:
    """Cell centres of a regular m x m grid on the unit square, (m*m, 2)."""
    c = (np.arange(m, dtype=np.float64) + 0.5) / m
    xx, yy = np.meshgrid(c, c, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def fibonacci_sphere(n: int) -> np.ndarray:
    """n Fibonacci points on the unit sphere, (n, 3)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def random_vector(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n)


@dataclass(frozen=True)
class Workload:
    """One product C = A*B on a point set, with the parameters of h2_build."""
    name: str
    points: np.ndarray = field(repr=False)
    kernel_a: KernelSpec
    kernel_b: KernelSpec
    eta: float          # admissible iff max(diam) <= eta * dist
    leaf_size: int
    order: int          # Chebyshev points per axis; rank k = order**dim
    eps: float

    @property
    def n(self) -> int:
        return self.points.shape[0]

    @property
    def dim(self) -> int:
        return self.points.shape[1]

    @property
    def k(self) -> int:
        return self.order ** self.dim


def plain_1d(n: int = 1024, eps: float = 1e-6, seed_offset: int = 0) -> Workload:
    """n uniform points on [0,1], -log|x-y| with diagonal 1, leaf 32,
    max(diam) <= 2 dist, order 4 (k = 4), C = A*A."""
    pts = uniform_points(n, 1, SEED_BASE + seed_offset)
    return Workload(f"plain1d_n{n}", pts, LOG, LOG, 2.0, 32, 4, eps)


def grid_2d(m: int = 128, eps: float = 1e-6) -> Workload:
    """m x m grid on the unit square, A = -log|x-y|/(2 pi) (diag 1),
    B = exp(-|x-y|^2/0.1), leaf 64, eta 2, order 4 (k = 16), C = A*B."""
    return Workload(f"grid2d_n{m * m}", grid_points(m), LOG_2PI, GAUSS_01, 2.0, 64, 4, eps)


def sphere_3d(n: int = 65536, eps: float = 1e-6) -> Workload:
    """Fibonacci sphere, 1/(4 pi |x-y|) (diag 0), leaf 64, eta 2, order 4 (k=64), C = A*A."""
    return Workload(f"sphere3d_n{n}", fibonacci_sphere(n), INV_4PI, INV_4PI, 2.0, 64, 4, eps)


def cube_3d(n: int, seed: int, eps: float = 1e-6, leaf: int = 64, order: int = 4) -> Workload:
    """n uniform points in the unit cube, A = 1/|x-y| (diag 0), B = exp(-|x-y|)."""
    return Workload(f"cube3d_n{n}", uniform_points(n, 3, seed), INV, EXP, 2.0, leaf, order, eps)


def square_2d(n: int, seed: int, eps: float = 1e-6, leaf: int = 64, order: int = 4) -> Workload:
    """n uniform points in the unit square, A = -log|x-y| (diag 1), B = exp(-|x-y|^2/0.1)."""
    return Workload(f"square2d_n{n}", uniform_points(n, 2, seed), LOG, GAUSS_01, 2.0, leaf, order, eps)
