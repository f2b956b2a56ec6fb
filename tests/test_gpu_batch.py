"""The batching form (h2_batch_*): many products of different sizes, kernels,
dimensions and ranks in merged launches, persistent GEMM chains over the tree
levels fed by a device work queue, one CUDA graph per batch.

Checked: every product of the batch is bitwise equal to the same product run
alone through h2_mul (each keeps its own workspace, and the arithmetic of a
job does not depend on the launch it runs in), also after the autotuner has
pinned other kernel variants and grids; within 1e-10 block-relative of the
oracle with identical ranks; a wait that nothing satisfies ends after about a
second with H2_ETIMEOUT and leaves the library usable."""
import numpy as np
import pytest

from oracle import h2oracle as O
from paper_2403_01566_gb300 import inputs as I
from tests.oracle_cases import build_pair

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900, method="thread")]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2403_01566_gb300 import h2  # noqa: E402

WORKLOADS = [
    I.grid_2d(32, 1e-6),
    I.plain_1d(1000, 1e-4),
    I.square_2d(1500, seed=7, leaf=32, order=3),
    I.cube_3d(1200, seed=11, leaf=40, order=2, eps=1e-4),  # ranks up to 41 at 1e-6, above the cap of 32
    I.sphere_3d(2048, 1e-6),
    I.cube_3d(2048, seed=13, leaf=64, order=4),
]


def _operands():
    ops = []
    for w in WORKLOADS:
        A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
        B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
        ops.append((w, A, B))
    return ops


@pytest.fixture(scope="module")
def ops():
    return _operands()


@pytest.mark.parametrize("precision", [0, 4])
def test_batch_bitwise_equal_to_products_alone(ops, precision):
    # the workloads plus a second product of the first structure (B * A)
    prods = [(A, B, w.eps) for w, A, B in ops] + [(ops[0][2], ops[0][1], 1e-6)]
    batch = h2.Batch(prods, precision=precision)
    info = batch.info()
    assert info["chains"] >= 1
    for rep in range(2):  # two replays of the captured batch
        batch.run()
        for i, (A, B, eps) in enumerate(prods):
            alone = h2.mul(A, B, eps, precision=precision).to_dense()
            got = batch.result(i).to_dense()
            assert np.array_equal(got, alone), (i, rep, np.abs(got - alone).max())
    print(f"\nbatch of {len(prods)} products, precision {precision}: {info}")


def test_batch_matches_oracle(ops):
    batch = h2.Batch([(A, B, w.eps) for w, A, B in ops])
    batch.run()
    for i, (w, A, B) in enumerate(ops):
        X, Y = build_pair(w)
        res = O.multiply(X, Y, w.eps)
        Z = X.dense() @ Y.dense()
        Cg = batch.result(i).to_dense()
        Co = res.C.dense()
        worst = 0.0
        for b in O.block_leaves(res.C.blocks):
            ix = np.ix_(b.t.idx, b.s.idx)
            nz = np.linalg.norm(Z[ix], 2) or 1.0
            worst = max(worst, np.linalg.norm(Cg[ix] - Co[ix], 2) / nz)
        assert worst <= 1e-10, (w.name, worst)
        rr, rc = batch.result(i).ranks()
        assert list(rr) == [res.ranks_row[c.id] for c in O.all_clusters(X.rows)]
        assert list(rc) == [res.ranks_col[c.id] for c in O.all_clusters(Y.cols)]


def test_autotuned_batch_keeps_results(ops):
    prods = [(A, B, w.eps) for w, A, B in ops]
    batch = h2.Batch(prods)
    batch.run()
    before = [batch.result(i).to_dense() for i in range(len(prods))]
    batch.autotune()
    assert h2.tuning_table().count("\n") >= 1
    batch.run()
    for i in range(len(prods)):
        assert np.array_equal(batch.result(i).to_dense(), before[i])
    # a batch created after tuning uses the pinned choices
    again = h2.Batch(prods)
    again.run()
    for i in range(len(prods)):
        assert np.array_equal(again.result(i).to_dense(), before[i])


def test_batch_wait_cap_returns_etimeout(ops):
    w, A, B = ops[0]
    bad = h2.Batch([(A, B, w.eps), (B, A, w.eps)], test_unreachable_wait=True)
    with pytest.raises(h2.H2Error) as ei:
        bad.run()
    assert ei.value.code == h2.H2_ETIMEOUT
    bad.free()
    # the context stays usable: a product and a normal batch
    ref = h2.mul(A, B, w.eps).to_dense()
    good = h2.Batch([(A, B, w.eps)])
    good.run()
    assert np.array_equal(good.result(0).to_dense(), ref)
