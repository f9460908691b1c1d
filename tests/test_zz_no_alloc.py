"""The allocation-free sizing entry point, checked against the regular one.

spgemm_rowptr_noalloc serves callers that cannot call cudaMalloc at run
time (for example, when another framework's allocator owns all device
memory): it computes C's row pointer with scratch held in a fixed array
inside the library. Here its output is compared, through the C ABI, with the
row pointer that spgemm_symbolic + spgemm_numeric produce and with the CPU
oracle's row sizes and exclusive scan, on two calls in a row, so that
contents the array keeps from one call cannot leak into the next; and at
the edges: an A with no rows, an A with exactly the largest accepted number
of rows, and a B wide enough that the bitmap kernel takes two passes. This
file is collected last on purpose."""

import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2206_07244_gb300 as ops  # noqa: E402
from paper_2206_07244_gb300 import _abi  # noqa: E402

ops.build()


def _csr_in(m):
    rpt = torch.as_tensor(m.rpt).cuda()
    col = torch.as_tensor(m.col, dtype=torch.int32).cuda()
    s = _abi.CsrIn()
    s.rows, s.cols, s.nnz = m.rows, m.cols, m.nnz
    s.rpt, s.rpt_is_i64 = rpt.data_ptr(), 1 if rpt.dtype == torch.int64 else 0
    s.col = col.data_ptr() if m.nnz else None
    s.val = None
    return s, (rpt, col)


def _rowptr_noalloc(A, B):
    lib = _abi.lib()
    a, keep_a = _csr_in(A)
    b, keep_b = _csr_in(B)
    out = torch.full((A.rows + 1,), -1, dtype=torch.int64, device="cuda")
    nnz = ctypes.c_int64(-1)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.spgemm_rowptr_noalloc(ctypes.byref(a), ctypes.byref(b),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream),
                                   ctypes.byref(nnz))
    torch.cuda.synchronize()
    del keep_a, keep_b
    return rc, out.cpu().numpy(), nnz.value


def _rowptr_regular(A, B):
    with ops.Handle() as h:
        C = h.multiply(ops.CSR.from_workload(A), ops.CSR.from_workload(B))
        h.status()
        return C.rpt.cpu().numpy()


def _dense_row_case():
    K, N = 1500, 40000
    B = W.random_csr(K, N, 0.02, seed=31)
    r = np.concatenate([np.zeros(K, dtype=np.int64), np.arange(1, 300) % 7 + 1])
    c = np.concatenate([np.arange(K), np.arange(1, 300) * 5 % K])
    A = W._from_coo(8, K, r, c, np.ones(r.size))
    return A, B


@pytest.mark.parametrize("case", ["rmat", "dense_row", "laplace"])
def test_noalloc_rowptr_matches_regular_entry_point(case):
    if case == "rmat":
        A = B = W.rmat(14, 16, seed=7)
    elif case == "dense_row":
        A, B = _dense_row_case()
    else:
        A = B = W.laplacian_2d(64)
    want = _rowptr_regular(A, B)
    for _ in range(2):  # two calls in a row share the same scratch array
        rc, got, nnz = _rowptr_noalloc(A, B)
        assert rc == 0
        assert np.array_equal(got, want)
        assert nnz == want[-1]


def _rowptr_oracle(A, B):
    return oracle.exclusive_scan(oracle.symbolic(A, B))


@pytest.mark.parametrize("case", ["rmat", "dense_row"])
def test_noalloc_rowptr_matches_oracle(case):
    A, B = (W.rmat(13, 8, seed=9),) * 2 if case == "rmat" else _dense_row_case()
    want = _rowptr_oracle(A, B)
    for _ in range(2):
        rc, got, nnz = _rowptr_noalloc(A, B)
        assert rc == 0
        assert np.array_equal(got, want)
        assert nnz == want[-1]


def test_noalloc_empty_a():
    A = W.Csr(0, 16, np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    B = W.rmat(4, 4, seed=1)
    for _ in range(2):
        rc, got, nnz = _rowptr_noalloc(A, B)
        assert rc == 0 and got.tolist() == [0] and nnz == 0


def test_noalloc_largest_accepted_size():
    # exactly SPGEMM_NOALLOC_MAX_ROWS rows (fills the bins and tile-sum
    # regions of the fixed array) with a few non-zeros
    n = 1 << 20
    rng = np.random.default_rng(41)
    rows = np.sort(rng.choice(n, 3000, replace=False))
    A = W._from_coo(n, 64, rows, rng.integers(0, 64, rows.size), np.ones(rows.size))
    B = W.random_csr(64, 5000, 0.05, seed=42)
    want = _rowptr_oracle(A, B)
    rc, got, nnz = _rowptr_noalloc(A, B)
    assert rc == 0 and np.array_equal(got, want) and nnz == want[-1]


def test_noalloc_columns_past_one_bitmap_pass():
    # 3M columns: the symbolic bitmap kernel covers them in two passes
    rng = np.random.default_rng(43)
    K, N = 40, 3_000_000
    br = np.repeat(np.arange(K), 6000)
    bc = np.concatenate([np.sort(rng.choice(N, 6000, replace=False)) for _ in range(K)])
    B = W._from_coo(K, N, br, bc, np.ones(bc.size))
    A = W._from_coo(4, K, np.repeat(np.arange(4), K), np.tile(np.arange(K), 4), np.ones(4 * K))
    want = _rowptr_oracle(A, B)
    for _ in range(2):
        rc, got, nnz = _rowptr_noalloc(A, B)
        assert rc == 0 and np.array_equal(got, want) and nnz == want[-1]


def test_noalloc_rejects_too_many_rows():
    n = (1 << 20) + 1
    A = W.Csr(n, 4, np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    B = W.Csr(4, 4, np.zeros(5, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    rc, _, _ = _rowptr_noalloc(A, B)
    assert rc == -1   # SPGEMM_ERR_INVALID
