"""Serving with continuous batching (h2_server_*): products of different
sizes, tolerances and structures submitted together run concurrently on the
server's streams; every result must be bitwise the same as the same product
run alone through h2_mul, and within its eps of the exact product.  Also:
several products of one structure at once (further plan instances), a memory
budget too small for all at once (requests wait for memory), and shutdown
with requests still queued."""
import numpy as np
import pytest

from paper_2403_01566_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(240, method="thread")]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2403_01566_gb300 import h2  # noqa: E402


def _operands(w):
    return (h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order),
            h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order))


def _blockrel_to_exact(C, w, eps):
    """Largest ||C_b - (AB)_b||_2 / ||(AB)_b||_2 over the blocks of the oracle's
    block tree of the product, against the exact dense product."""
    from oracle import h2oracle as O
    from tests.oracle_cases import build_pair
    X, Y = build_pair(w)
    Z = X.dense() @ Y.dense()
    Cd = C.to_dense()
    tb = O.build_block_tree(X.rows, Y.cols, w.eta)
    worst = 0.0
    for b in O.block_leaves(tb):
        ix = np.ix_(b.t.idx, b.s.idx)
        nz = np.linalg.norm(Z[ix], 2) or 1.0
        worst = max(worst, np.linalg.norm(Cd[ix] - Z[ix], 2) / nz)
    return worst


@pytest.mark.parametrize("precision", [0, 2, 4])
def test_each_result_same_alone_and_in_the_mix(precision):
    ws = [(I.grid_2d(32), 1e-6), (I.grid_2d(64), 1e-4), (I.plain_1d(1024), 1e-6), (I.grid_2d(32), 1e-4),
          (I.cube_3d(1200, seed=11, leaf=40, order=2), 1e-4), (I.grid_2d(64), 1e-6)]
    ops = [_operands(w) for w, _ in ws]
    alone = [h2.mul(A, B, eps, precision=precision).to_dense() for (A, B), (_, eps) in zip(ops, ws)]
    srv = h2.Server(slots=4)
    tickets = [srv.submit(A, B, eps, precision=precision) for (A, B), (_, eps) in zip(ops, ws)]
    for i, (t, ref) in enumerate(zip(tickets, alone)):
        C, q, tot = srv.wait(t)
        assert tot >= q >= 0.0
        assert np.array_equal(C.to_dense(), ref)
        if i < 3:  # the bound claimed above, against the exact product
            w, eps = ws[i]
            assert _blockrel_to_exact(C, w, eps) <= eps
    srv.close()


def test_same_structure_runs_on_several_instances():
    w = I.grid_2d(64)
    A, B = _operands(w)
    ref = h2.mul(A, B, 1e-6).to_dense()
    srv = h2.Server(slots=3)
    tickets = [srv.submit(A, B, 1e-6) for _ in range(6)]
    for t in tickets:
        C, _, _ = srv.wait(t)
        assert np.array_equal(C.to_dense(), ref)
    srv.close()


def test_small_budget_makes_requests_wait():
    w = I.grid_2d(32)
    A, B = _operands(w)
    ref = h2.mul(A, B, 1e-6).to_dense()
    srv = h2.Server(slots=4, mem_budget=1)  # nothing fits beside a running product: one at a time
    tickets = [srv.submit(A, B, 1e-6) for _ in range(4)]
    qs = []
    for t in tickets:
        C, q, _ = srv.wait(t)
        qs.append(q)
        assert np.array_equal(C.to_dense(), ref)
    srv.close()
    assert max(qs) > 0.0


def test_shutdown_with_queued_requests():
    w = I.grid_2d(32)
    A, B = _operands(w)
    srv = h2.Server(slots=1)
    for _ in range(5):
        srv.submit(A, B, 1e-6)
    srv.close()  # drops what has not started, waits for the running one
