"""GPU parity of spgemm_numeric_values: the numeric phase run again over the
structure that a handle kept from its last numeric call, for new values of
A and B with the same structure (the repeated products of an iterative
setup). Each result is compared with the CPU oracle on the new values:
structure bit for bit, values within helpers.VALUE_RTOL, or bit for bit
where every partial sum is an exact integer."""

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

ops.build()

ERR_INVALID, ERR_STATE, ERR_INTERNAL = -1, -4, -7


def dev(m):
    return ops.CSR.from_arrays(m.rows, m.cols, m.rpt, m.col, m.val)


def revalue(m, seed, integer=False):
    """Same rpt and col (duplicates and column order included), new values."""
    rng = np.random.default_rng(seed)
    v = rng.integers(-4, 5, size=m.nnz).astype(np.float64) if integer else rng.uniform(-1, 1, m.nnz)
    return W.Csr(m.rows, m.cols, m.rpt.copy(), m.col.copy(), v)


def check(A, B, C, exact=False, r0=0, r1=None):
    rpt, col, val, ab = oracle.spgemm(A, B, r0, r1)
    g_rpt, g_col, g_val = C.numpy()
    assert np.array_equal(g_rpt, rpt), "row pointers differ"
    assert np.array_equal(g_col, col), "column indices differ"
    if exact:
        assert np.array_equal(g_val, val), "values differ (exact case)"
    else:
        assert_values_close(g_val, val, ab)


def numeric_only(kernel):
    """Default symbolic bins; every numeric row the kernel can take goes to it
    (None: the default configuration)."""
    cfg = ops.default_config()
    if kernel is None:
        return cfg
    table = ops.kernel_table(1)
    bitmap = len(table) - 1
    if kernel == bitmap:
        cfg["num_kernel"], cfg["num_range"] = [bitmap], [-1]
    else:
        cfg["num_kernel"], cfg["num_range"] = [kernel, bitmap], [table[kernel][3], -1]
    return cfg


def expect_error(code, fn, *args):
    with pytest.raises(ops.SpgemmError) as e:
        fn(*args)
    assert e.value.code == code


@pytest.mark.parametrize("kernel", [None] + list(range(len(ops.kernel_table(1)))))
def test_new_values_twice(kernel):
    """Two re-runs in a row on R-MAT n = 2^11 (power-law rows over several
    bins), each against the oracle on its own values."""
    A = W.rmat(11, 12, seed=61)
    with ops.Handle(numeric_only(kernel)) as h:
        C = h.multiply(dev(A), dev(A))
        h.status()
        check(A, A, C)
        for seed in (1, 2):
            A2 = revalue(A, seed)
            d2 = dev(A2)
            assert h.numeric_values(d2, d2, C) is C
            h.status()
            check(A2, A2, C)


def test_rectangular_integer_values_exact():
    """A*B with duplicate and unsorted entries in A, integer values: every
    partial sum is exact, so the new values must match bit for bit."""
    A = W.random_csr(300, 200, 0.05, seed=5, duplicates=True, unsorted=True, integer_values=True)
    B = W.random_csr(200, 150, 0.08, seed=6, integer_values=True)
    with ops.Handle() as h:
        C = h.multiply(dev(A), dev(B))
        A2, B2 = revalue(A, 7, integer=True), revalue(B, 8, integer=True)
        h.numeric_values(dev(A2), dev(B2), C)
        h.status()
        check(A2, B2, C, exact=True)


def test_bitmap_kernel_on_every_row():
    A = W.random_csr(400, 300, 0.03, seed=13, duplicates=True, unsorted=True)
    B = W.random_csr(300, 900, 0.03, seed=14)
    with ops.Handle(numeric_only(len(ops.kernel_table(1)) - 1)) as h:
        C = h.multiply(dev(A), dev(B))
        B2 = revalue(B, 15)
        h.numeric_values(dev(A), dev(B2), C)
        h.status()
        check(A, B2, C)


def test_galerkin_new_fine_operator():
    """A*P for the 7-point operator on 9^3 with new fine-grid values (the
    setup of a multigrid solve whose coefficients change)."""
    A, P, _ = W.galerkin_problem(9)
    with ops.Handle() as h:
        dP = dev(P)
        AP = h.multiply(dev(A), dP)
        A2 = revalue(A, 21, integer=True)
        h.numeric_values(dev(A2), dP, AP)
        h.status()
        check(A2, P, AP, exact=True)


def test_row_window():
    A = W.rmat(12, 8, seed=23)
    r0, r1 = 100, 1733
    with ops.Handle() as h:
        h.symbolic(dev(A), dev(A), r0, r1)
        C = h.numeric(dev(A), dev(A))
        A2 = revalue(A, 3)
        d2 = dev(A2)
        h.numeric_values(d2, d2, C)
        h.status()
        check(A2, A2, C, r0=r0, r1=r1)


def test_empty_product():
    A = W.random_csr(50, 40, 0.1, seed=1)
    Z = W.Csr(40, 30, np.zeros(41, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    with ops.Handle() as h:
        C = h.multiply(dev(A), dev(Z))
        assert C.nnz == 0
        h.numeric_values(dev(revalue(A, 2)), dev(Z), C)
        h.status()


def test_state_is_checked():
    A = W.rmat(10, 8, seed=31)
    dA = dev(A)
    other = dev(W.rmat(10, 6, seed=32))
    with ops.Handle() as h:
        C0 = h.multiply(dA, dA)
        h.status()
        with ops.Handle() as fresh:   # no numeric call yet
            expect_error(ERR_STATE, fresh.numeric_values, dA, dA, C0)
        expect_error(ERR_STATE, h.numeric_values, other, other, C0)     # other sizes
        short = ops.CSR(C0.rows, C0.cols, C0.rpt, C0.col[:-1], C0.val[:-1])
        expect_error(ERR_INVALID, h.numeric_values, dA, dA, short)      # not that C
        h.symbolic(dA, dA)                                              # bins overwritten
        expect_error(ERR_STATE, h.numeric_values, dA, dA, C0)
        C1 = h.numeric(dA, dA)
        h.numeric_values(dA, dA, C1)
        h.status()
        check(A, A, C1)
        h.set_config(h.get_config())                                    # kernels may change
        expect_error(ERR_STATE, h.numeric_values, dA, dA, C1)
        # a learned-mode product keeps no plain structure
        h.set_predictor(W.mlp_init(0), margin=0.25)
        h.set_mode("learned")
        C2 = h.multiply(dA, dA)
        expect_error(ERR_STATE, h.numeric_values, dA, dA, C2)
        h.status()


def test_changed_structure_is_reported_and_handle_recovers():
    """A with its columns permuted has the same sizes but another product
    structure: rows whose size no longer matches are reported by
    spgemm_status (every store stays inside its row), and the handle then
    multiplies correctly again."""
    A = W.rmat(11, 12, seed=41)
    perm = np.random.default_rng(4).permutation(A.cols).astype(np.int32)
    Ap = W.Csr(A.rows, A.cols, A.rpt.copy(), perm[A.col], A.val.copy())
    with ops.Handle() as h:
        C = h.multiply(dev(A), dev(A))
        h.status()
        h.numeric_values(dev(Ap), dev(Ap), C)
        expect_error(ERR_INTERNAL, h.status)
        check(Ap, Ap, h.multiply(dev(Ap), dev(Ap)))
        h.status()
