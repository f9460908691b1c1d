"""Parity at the full sizes of the two benchmark workloads that the other GPU
tests cover only in small:

- learned sizing (trained predictor) on a row slab of the held-out R-MAT
  n = 2^21, degree 32 (seed 2021): every row's size, sum of columns and sum
  of values against the oracle's row checksums, and the values of sampled
  rows, the heaviest among them, in full;
- the batch of 512 multigrid Galerkin products P^T (A P) (sides uniform in
  [8, 48], seed 0, every product with its own inputs) in one persistent
  launch: all 1,024 products against the oracle, bit for bit (integer
  values), and even sides also against the closed form 4 L7(s/2)."""

import json

import numpy as np
import pytest

import oracle
import workloads as W
from helpers import assert_values_close

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2206_07244_gb300 as ops  # noqa: E402
from paper_2206_07244_gb300 import learned  # noqa: E402
from paper_2206_07244_gb300.batch import Batch, galerkin_batch  # noqa: E402

ops.build()

SLAB = (1 << 20, (1 << 20) + 16384)   # rows of C the benchmark's learned leg times


def held_out_expectations():
    """A, the slab's row sizes from the oracle, and the rows to compare in
    full (60 seeded + the 4 heaviest), relative to the slab's first row."""
    A = W.rmat(21, 32, seed=2021)
    r0, r1 = SLAB
    sizes = oracle.symbolic(A, A, r0, r1, threads=oracle.max_threads())
    rng = np.random.default_rng(3)
    rows = sorted(set(rng.integers(0, r1 - r0, 60).tolist()) | set(np.argsort(sizes)[-4:].tolist()))
    return A, sizes, rows


def galerkin_expectations(sides):
    """Oracle A P and P^T (A P) for every distinct side."""
    want = {}
    for s in np.unique(sides):
        A, P, PT = W.galerkin_problem(int(s))
        ap = oracle.spgemm(A, P, with_abs=False)
        AP = W.Csr(A.rows, P.cols, ap[0], ap[1], ap[2])
        ac = oracle.spgemm(PT, AP, with_abs=False)
        want[int(s)] = (ap[:3], ac[:3])
    return want


def test_learned_sizing_held_out_rmat_2_21_slab():
    A, sizes, rows = held_out_expectations()
    r0, r1 = SLAB
    man = json.load(open(learned.MANIFEST))
    theta = np.load(learned.WEIGHTS)
    dA = ops.CSR.from_workload(A)
    cnt_o, cs_o, vs_o, ab_o = oracle.row_checksums(A, A, r0, r1, threads=oracle.max_threads())
    with ops.Handle() as h:
        h.set_predictor(theta, man["margin"])
        h.set_mode("learned")
        h.symbolic(dA, dA, r0, r1)
        C = h.numeric(dA, dA)
        h.status()
        assert h.learned_stats()["one_phase_rows"] > 0    # the prediction was used
        rpt = C.rpt.cpu().numpy()
        assert rpt[0] == 0
        assert np.array_equal(np.diff(rpt), sizes), "row sizes differ from the oracle"
        # every row of the slab: sizes, column sums, value sums
        from test_gpu_parity import device_row_checks
        device_row_checks(C, 0, cnt_o, cs_o, vs_o, ab_o, "held-out slab")
        for i in rows:
            s, e = int(rpt[i]), int(rpt[i + 1])
            _, ocol, oval, oab = oracle.spgemm(A, A, r0 + i, r0 + i + 1)
            assert np.array_equal(C.col[s:e].cpu().numpy(), ocol), f"row {r0 + i}"
            assert_values_close(C.val[s:e].cpu().numpy(), oval, oab, what=f"row {r0 + i}")


def test_galerkin_batch_512_products():
    sides = W.galerkin_sides(512, seed=0)
    n = len(sides)
    want = galerkin_expectations(sides)
    with ops.Handle() as h:
        As, Bs, dep, _ = galerkin_batch(h, sides, share_inputs=False)
        with Batch(h, As, Bs, dep) as b:
            b.run()
            b.sync()
            for i, s in enumerate(int(x) for x in sides):
                for C, (wrpt, wcol, wval) in ((b.result(i), want[s][0]), (b.result(n + i), want[s][1])):
                    rpt, col, val = C.numpy()
                    assert np.array_equal(rpt, wrpt), f"product {i} (side {s}): row pointers"
                    assert np.array_equal(col, wcol), f"product {i} (side {s}): columns"
                    assert np.array_equal(val, wval), f"product {i} (side {s}): values"
                if s % 2 == 0:
                    L = W.laplacian_3d_7pt(s // 2)
                    rpt, col, val = b.result(n + i).numpy()
                    assert np.array_equal(rpt, L.rpt.astype(np.int64))
                    assert np.array_equal(col, L.col)
                    assert np.array_equal(val, 4.0 * L.val)
