"""CPU oracle for the row-wise SpGEMM hot path (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The CUDA library never
imports, links or runs anything here, and this package imports nothing from
the CUDA library.

What each function computes, and the passage it follows:

- ``nprod``       Sec. 5 step 1 / Sec. 2.1.2: intermediate products per row.
- ``symbolic``    Sec. 2.2 and Algorithm 4: distinct column keys per row.
- ``spgemm``      Eq. 1-2, Algorithm 5 and the CSR layout of Sec. 2.1.1:
                  the full product with sorted unique columns, computed with a
                  dense accumulator (plain C, ``spgemm_oracle.c``).
- ``row_checksums`` order-free per-row summary for sizes whose C does not fit
                  in host memory.
- ``binning``     Sec. 5.1, Algorithms 1-3: a row goes to the first bin j
                  whose inclusive upper range r_range[j] is >= its size.
- ``exclusive_scan`` Sec. 5.3: C.rpt is the exclusive sum of the n_nz.
- ``compression_ratio`` Eq. 3.

The C part is compiled on first use with gcc (``-O2 -fopenmp
-ffp-contract=off``) into ``oracle/_build/``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spgemm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_ERR = {-1: "column index out of range", -2: "row pointer not monotone",
        -3: "out of host memory", -4: "row pointer disagrees with counts"}


def build(force: bool = False) -> str:
    """Compile the C oracle (idempotent). Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-std=c11", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            INT = ctypes.c_int
            lib.oracle_nprod.argtypes = [I64, I64, P, P, P, P]
            lib.oracle_symbolic.argtypes = [I64, I64, I64, I64, P, P, P, P, P, INT]
            lib.oracle_numeric.argtypes = [I64, I64, I64, I64, P, P, P, P, P, P,
                                           P, P, P, P, INT]
            lib.oracle_row_checksums.argtypes = [I64, I64, I64, I64, P, P, P, P,
                                                 P, P, P, P, P, P, INT]
            lib.oracle_check_csr.argtypes = [I64, I64, P, P]
            lib.oracle_max_threads.argtypes = []
            for f in (lib.oracle_nprod, lib.oracle_symbolic, lib.oracle_numeric,
                      lib.oracle_row_checksums, lib.oracle_check_csr,
                      lib.oracle_max_threads):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(m):
    """(rows, cols, rpt int64, col int32, val float64), contiguous."""
    return (int(m.rows), int(m.cols),
            np.ascontiguousarray(m.rpt, dtype=np.int64),
            np.ascontiguousarray(m.col, dtype=np.int32),
            np.ascontiguousarray(m.val, dtype=np.float64))


def _rc(rc: int):
    if rc != 0:
        raise ValueError(f"oracle: {_ERR.get(rc, rc)}")


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def check_csr(m) -> None:
    rows, cols, rpt, col, _ = _csr(m)
    _rc(_load().oracle_check_csr(rows, cols, _p(rpt), _p(col)))


def _check_shapes(A, B):
    if A.cols != B.rows:
        raise ValueError(f"shape mismatch: A is {A.rows}x{A.cols}, B is {B.rows}x{B.cols}")


def nprod(A, B) -> np.ndarray:
    """Intermediate products per row of C = A*B (int64, length A.rows)."""
    _check_shapes(A, B)
    M, K, arpt, acol, _ = _csr(A)
    _, _, brpt, _, _ = _csr(B)
    out = np.zeros(M, dtype=np.int64)
    _rc(_load().oracle_nprod(M, K, _p(arpt), _p(acol), _p(brpt), _p(out)))
    return out


def symbolic(A, B, r0: int = 0, r1: int | None = None, threads: int = 0) -> np.ndarray:
    """n_nz of rows [r0, r1) of C = A*B (int64)."""
    _check_shapes(A, B)
    M, K, arpt, acol, _ = _csr(A)
    _, N, brpt, bcol, _ = _csr(B)
    r1 = M if r1 is None else r1
    check_csr(A); check_csr(B)
    out = np.zeros(max(r1 - r0, 0), dtype=np.int64)
    _rc(_load().oracle_symbolic(r0, r1, K, N, _p(arpt), _p(acol), _p(brpt),
                                _p(bcol), _p(out), threads))
    return out


def exclusive_scan(x: np.ndarray) -> np.ndarray:
    """Length n+1 int64 array: out[0] = 0, out[i+1] = out[i] + x[i]."""
    out = np.zeros(x.size + 1, dtype=np.int64)
    acc = 0
    xs = np.asarray(x, dtype=np.int64)
    if xs.size <= 4096:
        for i, v in enumerate(xs.tolist()):
            acc += v
            out[i + 1] = acc
    else:
        np.cumsum(xs, out=out[1:])
    return out


def spgemm(A, B, r0: int = 0, r1: int | None = None, threads: int = 0,
           with_abs: bool = True):
    """Rows [r0, r1) of C = A*B as (rpt int64 [r1-r0+1], col int32, val
    float64, abs float64 or None). ``abs`` holds sum |a_ik*b_kj| per entry."""
    _check_shapes(A, B)
    M, K, arpt, acol, aval = _csr(A)
    _, N, brpt, bcol, bval = _csr(B)
    r1 = M if r1 is None else r1
    nnz = symbolic(A, B, r0, r1, threads)
    rpt = exclusive_scan(nnz)
    total = int(rpt[-1])
    col = np.empty(total, dtype=np.int32)
    val = np.empty(total, dtype=np.float64)
    ab = np.empty(total, dtype=np.float64) if with_abs else None
    _rc(_load().oracle_numeric(r0, r1, K, N, _p(arpt), _p(acol), _p(aval),
                               _p(brpt), _p(bcol), _p(bval), _p(rpt), _p(col),
                               _p(val), _p(ab) if with_abs else None, threads))
    return rpt, col, val, ab


def spgemm_csr(A, B):
    """C = A*B as a workloads-style object with rows/cols/rpt/col/val."""
    rpt, col, val, _ = spgemm(A, B, with_abs=False)

    class _C:
        pass
    c = _C()
    c.rows, c.cols, c.rpt, c.col, c.val = A.rows, B.cols, rpt, col, val
    return c


def row_checksums(A, B, r0: int = 0, r1: int | None = None, threads: int = 0):
    """Per row of [r0, r1): (count, sum of columns, sum of values in column
    order, sum over the row's intermediate products of |a_ik * b_kj|). The
    last is the scale of the value tolerance (every entry of the row within
    1e-12 of its own sum of |a*b|, so the row's value sum within 1e-12 of
    this, up to the rounding of the two row sums)."""
    _check_shapes(A, B)
    M, K, arpt, acol, aval = _csr(A)
    _, N, brpt, bcol, bval = _csr(B)
    r1 = M if r1 is None else r1
    n = max(r1 - r0, 0)
    cnt = np.zeros(n, dtype=np.int64)
    cs = np.zeros(n, dtype=np.int64)
    vs = np.zeros(n, dtype=np.float64)
    ab = np.zeros(n, dtype=np.float64)
    _rc(_load().oracle_row_checksums(r0, r1, K, N, _p(arpt), _p(acol), _p(aval),
                                     _p(brpt), _p(bcol), _p(bval), _p(cnt),
                                     _p(cs), _p(vs), _p(ab), threads))
    return cnt, cs, vs, ab


def binning(sizes: np.ndarray, ranges) -> dict:
    """Algorithms 1-3 (Sec. 5.1): row i goes to the first bin j with
    sizes[i] <= ranges[j] (the last range may be a huge sentinel). Returns
    the bin of each row, the bin sizes, their exclusive-sum offsets, the
    ``bins`` array (row ids grouped by bin, increasing inside a bin; the GPU
    may order rows inside a bin differently) and the maximum size."""
    sizes = np.asarray(sizes, dtype=np.int64)
    ranges = [int(r) for r in ranges]
    nb = len(ranges)
    bin_of = np.full(sizes.size, -1, dtype=np.int64)
    for j in range(nb):
        take = (bin_of < 0) & (sizes <= ranges[j])
        bin_of[take] = j
    if (bin_of < 0).any():
        raise ValueError("a size exceeds the last bin range")
    bin_size = np.array([(bin_of == j).sum() for j in range(nb)], dtype=np.int64)
    bin_offset = exclusive_scan(bin_size)[:-1]
    bins = np.concatenate([np.nonzero(bin_of == j)[0] for j in range(nb)]).astype(np.int64) \
        if sizes.size else np.zeros(0, dtype=np.int64)
    return {"bin_of": bin_of, "bin_size": bin_size, "bin_offset": bin_offset,
            "bins": bins, "max": int(sizes.max()) if sizes.size else 0}


def compression_ratio(total_nprod: int, total_nnz: int) -> float:
    """Eq. 3: total intermediate products over total non-zeros of C."""
    return float(total_nprod) / float(total_nnz) if total_nnz else float("nan")
