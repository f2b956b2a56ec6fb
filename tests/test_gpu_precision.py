"""The reduced- and mixed-precision forms of h2_mul against the FP64 oracle.

precision 1 (FP32 contractions), 2 (compensated FP32), 3 (tensor cores, 5
BF16 slices) and 4 (tensor cores with 7 BF16 slices on the 64 x 64 stages,
about FP64).

Precision 1: the accumulation phases and the coupling projection compute FP32 products with
FP32 sums; agglomeration, condensation, QR, SVD, rank decisions and norms stay
FP64.  Requirements checked:

- the per-block bound ||C_b - (AB)_b||_2 <= eps ||(AB)_b||_2 against the exact
  dense product, as for the FP64 form;
- agreement with the FP64 oracle within eps block-relative (both forms are
  within eps of the exact product; the FP32 rounding itself is ~1e-7);
- the error of each result against the oracle is printed (pytest -s).

The rank decisions see the FP32 rounding, so ranks may differ from the
oracle's by a few where a singular value sits near the threshold; they are
compared only loosely (within 25% per cluster).
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

CASES = [
    (I.plain_1d(1024), 1e-6),
    (I.grid_2d(64), 1e-6),
    (I.grid_2d(64), 1e-4),
    (I.sphere_3d(2048), 1e-6),
    (I.cube_3d(2048, seed=13, leaf=64, order=4), 1e-6),
]


def _blockrel(Cg, Co, Z, blocks):
    wo = wz = 0.0
    for b in O.block_leaves(blocks):
        ix = np.ix_(b.t.idx, b.s.idx)
        nz = np.linalg.norm(Z[ix], 2) or 1.0
        wo = max(wo, np.linalg.norm(Cg[ix] - Co[ix], 2) / nz)
        wz = max(wz, np.linalg.norm(Cg[ix] - Z[ix], 2) / nz)
    return wo, wz


@pytest.mark.parametrize("w,eps", CASES, ids=[f"{w.name}-{e:g}" for w, e in CASES])
def test_fp32_contractions_within_eps(w, eps):
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
    C32 = h2.mul(A, B, eps, precision=1)
    C64 = h2.mul(A, B, eps, precision=0)
    X, Y = build_pair(w)
    res = O.multiply(X, Y, eps)
    Z = X.dense() @ Y.dense()
    d_oracle, d_exact = _blockrel(C32.to_dense(), res.C.dense(), Z, res.C.blocks)
    d64, _ = _blockrel(C64.to_dense(), res.C.dense(), Z, res.C.blocks)
    print(f"\n{w.name} eps={eps:g}: FP32-contraction form vs oracle {d_oracle:.3e}, vs exact {d_exact:.3e}; "
          f"FP64 form vs oracle {d64:.3e}")
    assert d_exact <= eps, d_exact
    assert d_oracle <= eps, d_oracle
    assert d64 <= 1e-10, d64
    rr, rc = C32.ranks()
    ro = np.array([res.ranks_row[c.id] for c in O.all_clusters(X.rows)])
    co = np.array([res.ranks_col[c.id] for c in O.all_clusters(Y.cols)])
    assert np.all(np.abs(np.asarray(rr) - ro) <= np.maximum(2, 0.25 * ro))
    assert np.all(np.abs(np.asarray(rc) - co) <= np.maximum(2, 0.25 * co))


CASES_DF = [
    (I.plain_1d(1024), 1e-6),
    (I.grid_2d(64), 1e-6),
    (I.grid_2d(32), 1e-4),
    (I.sphere_3d(2048), 1e-6),
    (I.cube_3d(2048, seed=13, leaf=64, order=4), 1e-6),
]


@pytest.mark.parametrize("w,eps", CASES_DF, ids=[f"{w.name}-{e:g}" for w, e in CASES_DF])
def test_compensated_contractions_match_oracle(w, eps):
    """precision 2: compensated FP32 contractions (~1e-13) keep the FP64
    result: within 1e-10 of the oracle and identical ranks."""
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
    Cdf = h2.mul(A, B, eps, precision=2)
    X, Y = build_pair(w)
    res = O.multiply(X, Y, eps)
    Z = X.dense() @ Y.dense()
    d_oracle, d_exact = _blockrel(Cdf.to_dense(), res.C.dense(), Z, res.C.blocks)
    print(f"\n{w.name} eps={eps:g}: compensated form vs oracle {d_oracle:.3e}, vs exact {d_exact:.3e}")
    assert d_oracle <= 1e-10, d_oracle
    assert d_exact <= eps, d_exact
    rr, rc = Cdf.ranks()
    assert list(rr) == [res.ranks_row[c.id] for c in O.all_clusters(X.rows)]
    assert list(rc) == [res.ranks_col[c.id] for c in O.all_clusters(Y.cols)]


@pytest.mark.parametrize("w,eps", CASES_DF, ids=[f"{w.name}-{e:g}" for w, e in CASES_DF])
def test_tensor_core_slices_match_oracle(w, eps):
    """precision 4: the 64 x 64 GEMM stages on the tensor cores with 7 BF16
    slices per operand (exact FP32 diagonal sums, compensated accumulation),
    the others compensated FP32, keep the FP64 result: within 1e-10 of the
    oracle, within eps of the exact product, identical ranks; two runs are
    bitwise equal."""
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
    Ctc = h2.mul(A, B, eps, precision=4)
    X, Y = build_pair(w)
    res = O.multiply(X, Y, eps)
    Z = X.dense() @ Y.dense()
    Dtc = Ctc.to_dense()
    d_oracle, d_exact = _blockrel(Dtc, res.C.dense(), Z, res.C.blocks)
    print(f"\n{w.name} eps={eps:g}: tensor-core 7-slice form vs oracle {d_oracle:.3e}, vs exact {d_exact:.3e}")
    assert d_oracle <= 1e-10, d_oracle
    assert d_exact <= eps, d_exact
    rr, rc = Ctc.ranks()
    assert list(rr) == [res.ranks_row[c.id] for c in O.all_clusters(X.rows)]
    assert list(rc) == [res.ranks_col[c.id] for c in O.all_clusters(Y.cols)]
    assert np.array_equal(h2.mul(A, B, eps, precision=4).to_dense(), Dtc)


CASES_TC5 = [
    (I.plain_1d(1024), 1e-4),
    (I.grid_2d(64), 1e-4),
    (I.grid_2d(64), 1e-6),
    (I.square_2d(1500, seed=7, leaf=32, order=3), 1e-4),
    (I.cube_3d(2048, seed=13, leaf=64, order=4), 1e-4),
]


@pytest.mark.parametrize("w,eps", CASES_TC5, ids=[f"{w.name}-{e:g}" for w, e in CASES_TC5])
def test_tensor_core_5slice_within_eps(w, eps):
    """precision 3: every GEMM stage on the tensor cores with 5 BF16 slices
    (40 bits relative to the chunk's row and column maxima); QR, SVD, rank
    decisions and norms FP64.  Every admissible block stays within eps of the
    exact product and of the FP64 oracle."""
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
    Cb = h2.mul(A, B, eps, precision=3)
    X, Y = build_pair(w)
    res = O.multiply(X, Y, eps)
    Z = X.dense() @ Y.dense()
    d_oracle, d_exact = _blockrel(Cb.to_dense(), res.C.dense(), Z, res.C.blocks)
    rr, rc = Cb.ranks()
    ro = [res.ranks_row[c.id] for c in O.all_clusters(X.rows)]
    print(f"\n{w.name} eps={eps:g}: tensor-core 5-slice form vs oracle {d_oracle:.3e}, vs exact {d_exact:.3e}; "
          f"largest row rank {max(rr)} (oracle {max(ro)})")
    assert d_exact <= eps, d_exact
    assert d_oracle <= eps, d_oracle


def test_precision_values():
    w = I.plain_1d(256)
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    for bad in (-1, 5):
        with pytest.raises(h2.H2Error):
            h2.mul(A, A, 1e-6, precision=bad)
    # the FP64 and FP32 forms have separate cached plans
    C1 = h2.mul(A, A, 1e-6, precision=1)
    C0 = h2.mul(A, A, 1e-6, precision=0)
    assert np.isfinite(C1.to_dense()).all() and np.isfinite(C0.to_dense()).all()


def test_profile_kinds_and_tensor_core_subset():
    """h2_mul_profile: the product it returns equals h2_mul's; kind 8 repeats
    the tensor-core GEMM stages (a subset of kind 0 in launches, jobs and
    time) with the slice products they issue (S(S+1)/2 = 28 mma.sync
    m16n8k16 per 16 x 8 tile and k step), at a rate below the tensor cores'
    peak; the FP64 form issues none."""
    w = I.grid_2d(64)
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
    with pytest.raises(ValueError):
        h2.mul_profile(A, B, 1e-6, (h2.KernelProf * 8)(), precision=4)
    for prec in (0, 4):
        prof = (h2.KernelProf * h2.PROFILE_KINDS)()
        Cp = h2.mul_profile(A, B, 1e-6, prof, precision=prec)
        C = h2.mul(A, B, 1e-6, precision=prec)
        assert np.array_equal(Cp.to_dense(), C.to_dense())
        tc, gemm = prof[8], prof[0]
        if prec == 0:
            assert tc.launches == 0 and tc.flops == 0.0
            continue
        assert 0 < tc.launches <= gemm.launches and 0 < tc.jobs <= gemm.jobs
        assert 0.0 < tc.ms <= gemm.ms
        rate = tc.flops / (tc.ms / 1e3)  # slice products issued per second
        assert 1e12 < rate < 2.5e15, rate  # below the tensor cores' dense BF16 peak
        # every profiled kind's time is positive where it launched
        for k in range(h2.PROFILE_KINDS):
            if prof[k].launches:
                assert prof[k].ms > 0.0
