"""spgemm_multiply_host (operands in host memory, C computed in slabs and
streamed back in chunks) against the CPU oracle: several slabs and many
chunks, rectangular operands, int64 row pointers, and a sink that stops."""

import ctypes

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
from paper_2206_07244_gb300 import _abi  # noqa: E402

ops.build()


def host_in(m, rpt64=False):
    rpt = np.ascontiguousarray(m.rpt.astype(np.int64 if rpt64 else np.int32))
    col = np.ascontiguousarray(m.col.astype(np.int32))
    val = np.ascontiguousarray(m.val.astype(np.float64))
    s = _abi.CsrIn()
    s.rows, s.cols, s.nnz = m.rows, m.cols, col.size
    s.rpt, s.rpt_is_i64 = rpt.ctypes.data, 1 if rpt64 else 0
    s.col = col.ctypes.data if col.size else None
    s.val = val.ctypes.data if val.size else None
    return s, (rpt, col, val)


def multiply_host(A, B, chunk, rpt64=False, stop_after=None):
    lib = _abi.lib()
    a, keep_a = host_in(A, rpt64)
    b, keep_b = host_in(B, rpt64)
    parts = []

    def view(addr, ctype, count):
        return np.ctypeslib.as_array(ctypes.cast(addr, ctypes.POINTER(ctype)), shape=(count,)).copy()

    def sink(ctx, r0, rows, prpt, pcol, pval, n):
        rp = view(prpt, ctypes.c_int64, rows + 1)
        cl = view(pcol, ctypes.c_int32, n) if n else np.zeros(0, np.int32)
        vl = view(pval, ctypes.c_double, n) if n else np.zeros(0)
        parts.append((r0, rows, rp, cl, vl))
        return 1 if stop_after is not None and len(parts) >= stop_after else 0

    cb = _abi.SINK_FN(sink)
    nnz = ctypes.c_int64()
    with ops.Handle() as h:
        rc = lib.spgemm_multiply_host(h._h, ctypes.byref(a), ctypes.byref(b), chunk, cb, None,
                                      ctypes.byref(nnz))
    return rc, nnz.value, parts


def assemble(parts, rows):
    rpt = np.zeros(rows + 1, dtype=np.int64)
    cols, vals = [], []
    nxt = 0
    for r0, n, rp, cl, vl in parts:
        assert r0 == nxt, "chunks out of order"
        assert rp[-1] - rp[0] == cl.size
        rpt[r0 + 1:r0 + n + 1] = rp[1:]
        assert rp[0] == rpt[r0], "row pointers are not absolute"
        cols.append(cl)
        vals.append(vl)
        nxt = r0 + n
    assert nxt == rows
    return rpt, np.concatenate(cols), np.concatenate(vals)


def check(A, B, chunk, rpt64=False, min_parts=1):
    rc, nnz, parts = multiply_host(A, B, chunk, rpt64)
    assert rc == 0
    assert len(parts) >= min_parts
    rpt, col, val = assemble(parts, A.rows)
    want = oracle.spgemm(A, B)
    assert nnz == want[0][-1]
    assert np.array_equal(rpt, want[0]) and np.array_equal(col, want[1])
    assert_values_close(val, want[2], want[3])


def test_slabs_and_chunks_rmat():
    A = W.rmat(13, 16, seed=51)
    check(A, A, 1 << 20, min_parts=8)


def test_rectangular_and_int64():
    A = W.random_csr(3000, 2000, 0.01, seed=52, duplicates=True, unsorted=True)
    B = W.random_csr(2000, 5000, 0.01, seed=53)
    check(A, B, 1 << 20, rpt64=True)


def test_empty_rows_and_single_chunk():
    A = W.random_csr(500, 400, 0.02, seed=54)
    A.rpt[100:300] = A.rpt[100]
    B = W.random_csr(400, 300, 0.05, seed=55)
    check(A, B, 1 << 30)


def test_sink_can_stop():
    A = W.rmat(12, 16, seed=56)
    rc, _, parts = multiply_host(A, A, 1 << 20, stop_after=2)
    assert rc == -8 and len(parts) == 2    # SPGEMM_ERR_ABORTED
