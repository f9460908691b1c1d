"""GB300 (sm_103a) row-wise SpGEMM, C = A * B, in CSR with float64 values.

A thin Python binding over the C ABI in ``include/opsparse.h``: it marshals
torch CUDA tensors into the ABI's plain structs and hands the library a
torch-backed device allocator. Every step of the multiplication runs in the
library's CUDA kernels; there is no Python or CPU fallback, and importing
the library fails loudly if it has not been built (``build()``).
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import _abi
from ._abi import MAX_BINS, SpgemmError

__all__ = ["CSR", "Handle", "spgemm", "build", "kernel_table", "default_config",
           "SpgemmError", "MAX_BINS", "library_path"]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    from . import _buildlib as _b
    return _b.build(force=force, verbose=verbose)


def library_path() -> str:
    return _abi.LIB_PATH


@dataclass
class CSR:
    """CSR matrix held in torch tensors (device or host).

    rpt: int32 or int64 (rows+1); col: int32 (nnz); val: float64 (nnz)."""
    rows: int
    cols: int
    rpt: object
    col: object
    val: object

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @classmethod
    def from_arrays(cls, rows, cols, rpt, col, val, device="cuda"):
        import torch
        return cls(int(rows), int(cols),
                   torch.as_tensor(rpt).to(device),
                   torch.as_tensor(col, dtype=torch.int32).to(device),
                   torch.as_tensor(val, dtype=torch.float64).to(device))

    @classmethod
    def from_workload(cls, m, device="cuda"):
        """From an object with rows/cols/rpt/col/val numpy arrays."""
        return cls.from_arrays(m.rows, m.cols, m.rpt, m.col, m.val, device)

    def numpy(self):
        return (self.rpt.cpu().numpy(), self.col.cpu().numpy(), self.val.cpu().numpy())


def _csr_in(m: CSR, with_values: bool = True) -> _abi.CsrIn:
    import torch
    for name, t in (("rpt", m.rpt), ("col", m.col), ("val", m.val)):
        if t is not None and not t.is_cuda:
            raise ValueError(f"CSR.{name} must be a CUDA tensor")
    if m.rpt.dtype not in (torch.int32, torch.int64):
        raise ValueError("CSR.rpt must be int32 or int64")
    if m.col.dtype != torch.int32:
        raise ValueError("CSR.col must be int32")
    if m.val is not None and m.val.dtype != torch.float64:
        raise ValueError("CSR.val must be float64")
    for t in (m.rpt, m.col, m.val):
        if t is not None and not t.is_contiguous():
            raise ValueError("CSR arrays must be contiguous")
    if m.rpt.numel() != m.rows + 1:
        raise ValueError("CSR.rpt must have rows+1 entries")
    s = _abi.CsrIn()
    s.rows, s.cols, s.nnz = m.rows, m.cols, m.col.numel()
    s.rpt = m.rpt.data_ptr()
    s.rpt_is_i64 = 1 if m.rpt.dtype == torch.int64 else 0
    s.col = m.col.data_ptr() if m.col.numel() else None
    s.val = m.val.data_ptr() if (with_values and m.val is not None and m.val.numel()) else None
    return s


def kernel_table(phase: int):
    """[(threads_per_row, block, table, max_size)] of the symbolic (0) or
    numeric (1) kernels; max_size -1 marks the bitmap kernel."""
    return _abi.kernel_table(phase)


def default_config() -> dict:
    """The library's default bin configuration (needs a GPU for the bitmap
    capacity; ranges do not depend on it)."""
    h = Handle()
    try:
        return h.get_config()
    finally:
        h.close()


class Handle:
    """One library handle: scratch memory, side streams and the bin
    configuration. Output arrays are allocated with torch's caching allocator
    on the handle's stream (torch's current stream at creation)."""

    def __init__(self, config: dict | None = None, stream=None, torch_alloc: bool = True):
        import torch
        lib = _abi.lib()
        self._lib = lib
        self._device = torch.device("cuda", torch.cuda.current_device())
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        self._live = {}
        self._h = ctypes.c_void_p()
        if torch_alloc:
            def _alloc(nbytes, stream, ctx):
                try:
                    t = torch.empty(int(nbytes), dtype=torch.uint8, device=self._device)
                except RuntimeError:
                    return None
                p = t.data_ptr()
                self._live[p] = t
                return p

            def _free(ptr, stream, ctx):
                self._live.pop(ptr, None)

            self._alloc_cb = _abi.ALLOC_FN(_alloc)
            self._free_cb = _abi.FREE_FN(_free)
        else:
            self._alloc_cb = _abi.ALLOC_FN()
            self._free_cb = _abi.FREE_FN()
        cfg = _abi.config_from_dict(config) if config else None
        _abi.check(lib.spgemm_create(ctypes.byref(self._h),
                                     ctypes.byref(cfg) if cfg is not None else None,
                                     self._alloc_cb, self._free_cb, None,
                                     ctypes.c_void_p(self._stream.cuda_stream)),
                   "spgemm_create")
        self._torch_alloc = torch_alloc

    # -- configuration ----------------------------------------------------------
    def get_config(self) -> dict:
        c = _abi.Config()
        _abi.check(self._lib.spgemm_get_config(self._h, ctypes.byref(c)), "spgemm_get_config")
        return _abi.config_to_dict(c)

    def set_config(self, config: dict | None):
        c = _abi.config_from_dict(config) if config else None
        _abi.check(self._lib.spgemm_set_config(self._h, ctypes.byref(c) if c is not None else None),
                   "spgemm_set_config")

    # -- the two phases -----------------------------------------------------------
    def symbolic(self, A: CSR, B: CSR, row_begin: int = 0, row_end: int | None = None) -> int:
        row_end = A.rows if row_end is None else row_end
        a, b = _csr_in(A), _csr_in(B)   # values: the learned mode multiplies here
        nnz = ctypes.c_int64()
        _abi.check(self._lib.spgemm_symbolic(self._h, ctypes.byref(a), ctypes.byref(b),
                                             row_begin, row_end, ctypes.byref(nnz)),
                   "spgemm_symbolic")
        self._last = (row_begin, row_end)
        return int(nnz.value)

    def numeric(self, A: CSR, B: CSR, out: tuple | None = None) -> CSR:
        """Numeric phase of the last symbolic window. ``out`` = (col, val)
        tensors to write into (each with at least nnz entries)."""
        import torch
        a, b = _csr_in(A), _csr_in(B)
        c = _abi.CsrOut()
        if out is not None:
            c.col = out[0].data_ptr()
            c.val = out[1].data_ptr()
        _abi.check(self._lib.spgemm_numeric(self._h, ctypes.byref(a), ctypes.byref(b),
                                            ctypes.byref(c)), "spgemm_numeric")
        return self._wrap(c, out)

    def multiply(self, A: CSR, B: CSR) -> CSR:
        self.symbolic(A, B)
        return self.numeric(A, B)

    def numeric_values(self, A: CSR, B: CSR, C: CSR) -> CSR:
        """New values of C for A and B with the structure of the last
        ``numeric`` call (same rpt and col, new val): only the numeric kernels
        run, over the rows' kept bins. ``C`` is that call's result; its val
        (and, with the same columns, its col) is overwritten in place."""
        import torch
        a, b = _csr_in(A), _csr_in(B)
        if C.rpt.dtype != torch.int64 or not (C.rpt.is_cuda and C.col.is_cuda and C.val.is_cuda):
            raise ValueError("C must be a CUDA CSR with an int64 row pointer")
        c = _abi.CsrOut()
        c.rows, c.cols, c.nnz = C.rows, C.cols, C.nnz
        c.rpt = C.rpt.data_ptr()
        c.col = C.col.data_ptr() if C.nnz else None
        c.val = C.val.data_ptr() if C.nnz else None
        _abi.check(self._lib.spgemm_numeric_values(self._h, ctypes.byref(a), ctypes.byref(b),
                                                   ctypes.byref(c)), "spgemm_numeric_values")
        return C

    def _wrap(self, c: _abi.CsrOut, out) -> CSR:
        import torch
        rows, nnz = int(c.rows), int(c.nnz)
        if not self._torch_alloc:
            raise RuntimeError("outputs of a handle without torch_alloc are raw pointers; "
                               "use the C ABI directly")
        rpt = self._live.pop(c.rpt).view(torch.int64)[: rows + 1]
        if out is None:
            col = self._live.pop(c.col).view(torch.int32)[:nnz]
            val = self._live.pop(c.val).view(torch.float64)[:nnz]
        else:
            col, val = out[0][:nnz], out[1][:nnz]
        return CSR(rows, int(c.cols), rpt, col, val)

    # -- learned sizing ------------------------------------------------------------
    def set_predictor(self, theta, margin: float = 0.25):
        """theta: 4673 float32 parameters (torch CUDA tensor or numpy array)."""
        import numpy as np
        import torch
        t = theta if isinstance(theta, torch.Tensor) else torch.as_tensor(np.asarray(theta, np.float32))
        t = t.to(dtype=torch.float32, device=self._device).contiguous()
        _abi.check(self._lib.spgemm_set_predictor(self._h, ctypes.c_void_p(t.data_ptr()),
                                                  ctypes.c_float(margin)), "spgemm_set_predictor")
        torch.cuda.current_stream().synchronize()

    def set_mode(self, mode: str):
        m = {"plain": 0, "learned": 1}[mode]
        _abi.check(self._lib.spgemm_set_mode(self._h, m), "spgemm_set_mode")

    def learned_stats(self) -> dict:
        n = 6 + MAX_BINS
        arr = (ctypes.c_int64 * n)()
        _abi.check(self._lib.spgemm_learned_stats(self._h, arr, n), "spgemm_learned_stats")
        return {"one_phase_rows": arr[0], "mispredicted_rows": arr[1], "exact_rows": arr[2],
                "temp_entries": arr[3], "rows_over_3_4_full": arr[4],
                "rows_fit_smaller_table": arr[5], "factor_log2": list(arr[6:n])}

    # -- diagnostics -------------------------------------------------------------
    def stats(self) -> dict:
        n = 4 + 2 * MAX_BINS
        arr = (ctypes.c_int64 * n)()
        _abi.check(self._lib.spgemm_last_stats(self._h, arr, n), "spgemm_last_stats")
        v = list(arr)
        return {"total_nprod": v[0], "max_nprod": v[1], "total_nnz": v[2], "max_nnz": v[3],
                "sym_bins": v[4:4 + MAX_BINS], "num_bins": v[4 + MAX_BINS:]}

    def window_stats(self) -> dict:
        arr = (ctypes.c_int64 * 9)()
        _abi.check(self._lib.spgemm_window_stats(self._h, arr, 9), "spgemm_window_stats")
        v = list(arr)
        return {"planned": bool(v[0]), "used": bool(v[1]), "windows": v[2], "column_windows": v[3],
                "cell_log2": v[4], "cells": v[5], "budget": v[6], "whole_width_max": v[7],
                "split": bool(v[8])}

    PHASES = ("bitmap_clear", "pass1_columns", "prefix_counts", "ccol_write", "cval_clear",
              "pass2_reductions", "priority_reset")

    def set_phase_clocks(self, enable: bool) -> None:
        """Per-phase SM clock sums of the numeric bitmap kernel (profiling)."""
        _abi.check(self._lib.spgemm_set_phase_clocks(self._h, int(bool(enable))), "spgemm_set_phase_clocks")

    def bitmap_phase_clocks(self, reset: bool = True) -> dict:
        arr = (ctypes.c_int64 * len(self.PHASES))()
        _abi.check(self._lib.spgemm_bitmap_phase_clocks(self._h, arr, len(self.PHASES), int(bool(reset))),
                   "spgemm_bitmap_phase_clocks")
        return dict(zip(self.PHASES, list(arr)))

    def status(self) -> None:
        _abi.check(self._lib.spgemm_status(self._h), "spgemm_status")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.spgemm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


_default = None


def spgemm(A: CSR, B: CSR, handle: Handle | None = None) -> CSR:
    """C = A * B on the GPU (two-phase, Sec. 2.2)."""
    global _default
    if handle is None:
        if _default is None:
            _default = Handle()
        handle = _default
    return handle.multiply(A, B)
