"""CPU test of the planner (host logic): the stage lists that the CUDA
kernels execute, run by a plain CPU interpreter of the stage semantics
(tests/host/stage_interpreter.cpp), must reproduce the oracle's product:
within 1e-10 block-relative (the FP64 tolerance) with identical adaptive
ranks, on 1D, 2D, 3D and ragged cases, and for the H-matrix output variant
against the oracle's pre-recompression factors.  No GPU is involved; the
interpreter links only the planner and the host tree / Chebyshev code."""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

from oracle import h2oracle as O
from paper_2403_01566_gb300 import inputs as I
from tests.oracle_cases import build_pair

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2403_01566_gb300", "csrc")


@pytest.fixture(scope="session")
def interpreter(tmp_path_factory):
    gxx = shutil.which("g++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not gxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("interp") / "stage_interpreter")
    cmd = [gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe,
           os.path.join(ROOT, "tests", "host", "stage_interpreter.cpp"),
           os.path.join(ROOT, "tests", "host", "host_assembly.cpp"),
           os.path.join(CSRC, "h2_plan.cpp"), os.path.join(CSRC, "h2_build.cpp"),
           "-I", os.path.join(ROOT, "include"), "-I", cuda_inc]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def run_interpreter(exe, w, eps, tmp_path, hmatrix=False, max_rank=0, svd_sweeps=None, expect_rc=0):
    pts = tmp_path / "pts.bin"
    out = tmp_path / "out.bin"
    np.ascontiguousarray(w.points, dtype=np.float64).tofile(pts)
    ka, kb = w.kernel_a, w.kernel_b
    args = [exe, str(pts), str(w.n), str(w.dim), str(w.leaf_size), str(w.order), repr(w.eta), repr(eps),
            str(ka.kind), repr(ka.scale), repr(ka.diag), repr(ka.width),
            str(kb.kind), repr(kb.scale), repr(kb.diag), repr(kb.width), str(max_rank), "1" if hmatrix else "0",
            str(out)]
    if svd_sweeps is not None:
        args.append(str(svd_sweeps))
    r = subprocess.run(args, capture_output=True, text=True, timeout=600)
    if expect_rc != 0:
        assert r.returncode == expect_rc, r.stderr[-2000:]
        return r.stderr
    assert r.returncode == 0, r.stderr[-2000:]
    raw = np.fromfile(out, dtype=np.uint8)
    n = w.n
    D = np.frombuffer(raw[:8 * n * n].tobytes(), dtype=np.float64).reshape(n, n)
    ranks = np.frombuffer(raw[8 * n * n:].tobytes(), dtype=np.int32)
    stats = {ln.split()[1]: int(ln.split()[2]) for ln in r.stdout.splitlines() if ln.startswith("stat ")}
    return D, ranks, stats


def worst_blockrel(D, Dref, Z, blocks):
    worst = 0.0
    for b in O.block_leaves(blocks):
        ix = np.ix_(b.t.idx, b.s.idx)
        nz = np.linalg.norm(Z[ix], 2) or 1.0
        worst = max(worst, np.linalg.norm(D[ix] - Dref[ix], 2) / nz)
    return worst


CASES = [
    (I.grid_2d(32), 1e-6),
    (I.plain_1d(1000), 1e-4),                     # ragged leaves
    (I.square_2d(1500, seed=7, leaf=32, order=3), 1e-6),
    (I.cube_3d(1200, seed=11, leaf=40, order=2), 1e-4),
    # k = 64: the widest agglomeration merges exceed the SVD's shared memory
    # and take the second-QR route, and some condensed QRs stop at the noise
    # floor
    (I.sphere_3d(2048), 1e-6),
]


@pytest.mark.parametrize("w,eps", CASES, ids=[f"{w.name}-{e:g}" for w, e in CASES])
def test_planned_stages_reproduce_the_oracle(interpreter, tmp_path, w, eps):
    D, ranks, stats = run_interpreter(interpreter, w, eps, tmp_path)
    # launch limits the kernels are configured for: k_qr 96 KB (128-row TSQR
    # chunks of 64 columns), k_svd 76 KB (SVD_SMEM_DOUBLES), k_norm n <= 128
    assert stats["smem_max_qr"] <= 8 * (64 + 128) * 64
    assert stats["smem_max_svd"] <= 8 * 9732
    assert stats["norm_max_n"] <= 128
    if w.dim == 3 and w.order == 4:
        assert stats.get("agg_two_step", 0) > 0
        assert stats.get("qr_truncated", 0) > 0
    # every agglomerated block takes ||G_b||_2 from the SVD of its last merge
    # (Section 5.3 weights), not from a norm job of its own
    assert stats.get("norms_from_agglomeration", 0) == stats.get("agglomerated", 0)
    X, Y = build_pair(w)
    res = O.multiply(X, Y, eps)
    Z = X.dense() @ Y.dense()
    assert worst_blockrel(D, res.C.dense(), Z, res.C.blocks) <= 1e-10
    ncl = len(ranks) // 2
    assert list(ranks[:ncl]) == [res.ranks_row[c.id] for c in O.all_clusters(X.rows)]
    assert list(ranks[ncl:]) == [res.ranks_col[c.id] for c in O.all_clusters(Y.cols)]


def test_planned_hmatrix_variant_reproduces_the_oracle_factors(interpreter, tmp_path):
    w = I.grid_2d(32)
    D, _, _ = run_interpreter(interpreter, w, 1e-6, tmp_path, hmatrix=True)
    X, Y = build_pair(w)
    res = O.multiply(X, Y, 1e-6)
    Do = res.C.dense()
    for b in O.block_leaves(res.C.blocks):
        if b.adm:
            L, R = res.factors[id(b)]
            Do[np.ix_(b.t.idx, b.s.idx)] = L @ R.T
    Z = X.dense() @ Y.dense()
    assert worst_blockrel(D, Do, Z, res.C.blocks) <= 1e-10


def test_svd_sweep_cap_reports_nonconvergence(interpreter, tmp_path):
    """The sweep cap of the Jacobi SVDs is a per-product parameter: one sweep
    cannot diagonalise the wide agglomeration merges, so the stage semantics
    report the non-convergence code -5 (H2_ENOCONV at the C ABI) instead of
    iterating on; with the default cap the same product converges."""
    w = I.grid_2d(32)
    err = run_interpreter(interpreter, w, 1e-6, tmp_path, svd_sweeps=1, expect_rc=4)
    assert "interpreter error -5" in err
    run_interpreter(interpreter, w, 1e-6, tmp_path, svd_sweeps=0)


@pytest.mark.parametrize("w", [I.plain_1d(256), I.grid_2d(16)], ids=lambda w: w.name)
def test_planned_exact_product_at_eps0(interpreter, tmp_path, w):
    """eps = 0 keeps every nonzero singular value: the planned stages give
    A*B to rounding in every block of the oracle's target block tree."""
    D, _, _ = run_interpreter(interpreter, w, 0.0, tmp_path, max_rank=64)
    X, Y = build_pair(w)
    Z = X.dense() @ Y.dense()
    assert worst_blockrel(D, Z, Z, O.build_block_tree(X.rows, Y.cols, w.eta)) <= 1e-12


def test_planned_single_leaf_tree(interpreter, tmp_path):
    """n <= leaf size: the root is a leaf and C is one dense block."""
    w = I.plain_1d(20)
    D, _, _ = run_interpreter(interpreter, w, 1e-6, tmp_path)
    X, Y = build_pair(w)
    Z = X.dense() @ Y.dense()
    assert np.max(np.abs(D - Z)) <= 1e-13 * np.abs(Z).max()
