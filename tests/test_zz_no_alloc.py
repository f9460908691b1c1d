"""The allocation-free sizing entry point, checked against the regular one.

spgemm_rowptr_noalloc serves callers that cannot call cudaMalloc at run
time (for example, when another framework's allocator owns all device
memory): it computes C's row pointer with scratch held in a fixed array
inside the library. Here its output is compared, through the C ABI, with the
row pointer that spgemm_symbolic + spgemm_numeric produce, on two calls in a
row, so that contents the array keeps from one call cannot leak into the
next. This file is collected last on purpose."""

import ctypes

import numpy as np
import pytest

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


def test_noalloc_rejects_too_many_rows():
    n = (1 << 20) + 1
    A = W.Csr(n, 4, np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    B = W.Csr(4, 4, np.zeros(5, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    rc, _, _ = _rowptr_noalloc(A, B)
    assert rc == -1   # SPGEMM_ERR_INVALID
