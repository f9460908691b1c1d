"""Batched products (one persistent launch under a CUDA graph) against the
oracle: multigrid Galerkin chains P^T (A P), where every product of the
batch is checked (even sides also against the closed form 4 L7(s/2)), and
independent random products; graph replays; and a bounded wait that runs
out and is reported as SPGEMM_ERR_TIMEOUT."""

import numpy as np
import pytest

import oracle
import workloads as W
from helpers import assert_values_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2206_07244_gb300 as ops  # noqa: E402
from paper_2206_07244_gb300.batch import Batch, galerkin_batch  # noqa: E402

ops.build()


def _np(C):
    return C.numpy()


def test_galerkin_batch_every_product():
    sides = [4, 5, 8, 9, 12, 13, 16, 7, 6, 11, 10, 15]
    with ops.Handle() as h:
        As, Bs, dep, _ = galerkin_batch(h, sides)
        with Batch(h, As, Bs, dep) as b:
            b.run()
            b.sync()
            n = len(sides)
            for i, s in enumerate(sides):
                A, P, PT = W.galerkin_problem(s)
                rpt, col, val = _np(b.result(i))
                want = oracle.spgemm(A, P)
                assert np.array_equal(rpt, want[0]) and np.array_equal(col, want[1])
                assert np.array_equal(val, want[2])          # integers: exact
                APo = oracle.spgemm_csr(A, P)
                rpt2, col2, val2 = _np(b.result(n + i))
                want2 = oracle.spgemm(PT, W.Csr(APo.rows, APo.cols, APo.rpt, APo.col, APo.val))
                assert np.array_equal(rpt2, want2[0]) and np.array_equal(col2, want2[1])
                assert np.array_equal(val2, want2[2])
                if s % 2 == 0:
                    L = W.laplacian_3d_7pt(s // 2)
                    assert np.array_equal(col2, L.col) and np.array_equal(val2, 4.0 * L.val)


def test_independent_products_and_replay():
    mats = [(W.random_csr(200 + 10 * i, 150, 0.03, seed=i, duplicates=True, unsorted=True),
             W.random_csr(150, 120 + i, 0.04, seed=50 + i)) for i in range(9)]
    with ops.Handle() as h:
        As = [ops.CSR.from_workload(a) for a, _ in mats]
        Bs = [ops.CSR.from_workload(b) for _, b in mats]
        with Batch(h, As, Bs) as b:
            for rep in range(3):   # graph replays give the same products
                b.run()
                b.sync()
                for i, (A, B) in enumerate(mats):
                    rpt, col, val = _np(b.result(i))
                    want = oracle.spgemm(A, B)
                    assert np.array_equal(rpt, want[0]) and np.array_equal(col, want[1])
                    assert_values_close(val, want[2], want[3])


@pytest.mark.parametrize("variant,tiny", [(0, True), (0, False), (1, False), (2, False)])
def test_each_kernel_variant(variant, tiny):
    # tiny=False sends the A P products (at most 7 products per row) through
    # the hash tables as well
    sides = [6, 9, 14]
    with ops.Handle() as h:
        As, Bs, dep, _ = galerkin_batch(h, sides)
        with Batch(h, As, Bs, dep, variant=variant, tile_rows=64, tiny=tiny) as b:
            b.run()
            b.sync()
            assert b.info()["table"] in (64, 128, 256)
            for i, s in enumerate(sides):
                A, P, PT = W.galerkin_problem(s)
                APo = oracle.spgemm_csr(A, P)
                rpt, col, val = _np(b.result(i))
                assert np.array_equal(rpt, APo.rpt) and np.array_equal(col, APo.col)
                assert np.array_equal(val, APo.val)
                want = oracle.spgemm(PT, W.Csr(APo.rows, APo.cols, APo.rpt, APo.col, APo.val))
                rpt, col, val = _np(b.result(len(sides) + i))
                assert np.array_equal(col, want[1]) and np.array_equal(val, want[2])


def test_tile_rows_limit():
    A = W.random_csr(100, 50, 0.1, seed=3)
    B = W.random_csr(50, 40, 0.1, seed=4)
    with ops.Handle() as h:
        with pytest.raises(ops.SpgemmError):
            Batch(h, [ops.CSR.from_workload(A)], [ops.CSR.from_workload(B)], tile_rows=2048)


def test_rows_too_large_are_rejected():
    A = W.random_csr(10, 400, 0.9, seed=1)
    B = W.random_csr(400, 300, 0.5, seed=2)
    with ops.Handle() as h:
        with pytest.raises(ops.SpgemmError) as e:
            Batch(h, [ops.CSR.from_workload(A)], [ops.CSR.from_workload(B)])
        assert e.value.code == -1


def test_bounded_wait_reports_timeout():
    # A large product (108 row tiles of 1024 rows) and a product that depends
    # on it: its scan item is taken while the tiles are still running, and a
    # wait limit of one poll runs out.
    big = W.laplacian_3d_7pt(48)
    P = W.aggregation_prolongator(48)
    PT = W.transpose(P)
    with ops.Handle() as h:
        dA, dP, dPT = (ops.CSR.from_workload(m) for m in (big, P, PT))
        with Batch(h, [dA, dPT], [dP, None], [-1, 0], tile_rows=1024, spin_limit=1) as b:
            b.run()
            with pytest.raises(ops.SpgemmError) as e:
                b.sync()
            assert e.value.code == -5   # SPGEMM_ERR_TIMEOUT
        h.status()
        # the handle stays usable
        C = h.multiply(dA, dP)
        h.status()
        assert C.nnz > 0
