"""Batched products in one persistent, graph-captured launch (argument
marshalling over spgemm_batch_* of include/opsparse.h)."""

from __future__ import annotations

import ctypes

from . import CSR, Handle, _abi, _csr_in


class Batch:
    """C_i = A_i * B_i for a list of products; B_i may be the C of an earlier
    product j (b_from[i] = j). Inputs must stay alive while the batch does."""

    def __init__(self, handle: Handle, As, Bs, b_from=None, variant: int = -1, tile_rows: int = 0,
                 spin_limit: int = 0, tiny: bool = True):
        import torch
        n = len(As)
        self._h = handle
        self._keep = (list(As), list(Bs))
        Arr = _abi.CsrIn * max(n, 1)
        a, bb = Arr(), Arr()
        for i in range(n):
            a[i] = _csr_in(As[i])
            if Bs[i] is not None:
                bb[i] = _csr_in(Bs[i])
        dep = (ctypes.c_int32 * max(n, 1))(*([(-1 if b_from is None else int(b_from[i])) for i in range(n)]
                                              or [0]))
        opt = _abi.BatchOptions(variant, tile_rows, spin_limit, 0 if tiny else 1, 0)
        self._b = ctypes.c_void_p()
        lib = _abi.lib()
        self._lib = lib
        _abi.check(lib.spgemm_batch_create(ctypes.byref(self._b), handle._h, n, a, bb, dep,
                                           ctypes.byref(opt)), "spgemm_batch_create")
        self.n = n
        self._torch = torch

    def run(self):
        _abi.check(self._lib.spgemm_batch_run(self._b), "spgemm_batch_run")

    def sync(self):
        _abi.check(self._lib.spgemm_batch_sync(self._b), "spgemm_batch_sync")

    def info(self) -> dict:
        arr = (ctypes.c_int64 * 6)()
        _abi.check(self._lib.spgemm_batch_info(self._b, arr, 6), "spgemm_batch_info")
        keys = ("products", "items", "blocks", "lanes_per_row", "table", "tile_rows")
        return dict(zip(keys, list(arr)))

    def _view(self, ptr: int, count: int, dtype):
        """Tensor view of `count` elements at device address ptr inside one
        of the handle's allocations."""
        torch = self._torch
        for base, t in self._h._live.items():
            if base <= ptr < base + t.numel():
                off = ptr - base
                size = torch.tensor([], dtype=dtype).element_size()
                return t[off:off + count * size].view(dtype)
        raise RuntimeError("result pointer outside the handle's allocations")

    def result(self, i: int) -> CSR:
        torch = self._torch
        c = _abi.CsrOut()
        _abi.check(self._lib.spgemm_batch_result(self._b, i, ctypes.byref(c)), "spgemm_batch_result")
        rows, nnz = int(c.rows), int(c.nnz)
        return CSR(rows, int(c.cols), self._view(c.rpt, rows + 1, torch.int64),
                   self._view(c.col, nnz, torch.int32), self._view(c.val, nnz, torch.float64))

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            self._lib.spgemm_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def galerkin_batch(handle: Handle, sides, device="cuda", share_inputs: bool = True):
    """Inputs of the products A_s P_s and P_s^T (A_s P_s) of every side s:
    (As, Bs, b_from, inputs), products 0..n-1 the A P of each side and n..2n-1
    the P^T (A P), whose B is product i - n. With share_inputs one set of
    device matrices serves every product of the same side; without it every
    product reads its own copy (as distinct operators would). `inputs[i]` is
    the (A, P, P^T) of side i."""
    import workloads as W
    host = {}
    for s in sides:
        s = int(s)
        if s not in host:
            host[s] = W.galerkin_problem(s)
    dev_cache = {}
    inputs = []
    for s in sides:
        s = int(s)
        if share_inputs and s in dev_cache:
            inputs.append(dev_cache[s])
            continue
        trip = tuple(CSR.from_workload(m, device) for m in host[s])
        dev_cache[s] = trip
        inputs.append(trip)
    n = len(sides)
    As = [inputs[i][0] for i in range(n)] + [inputs[i][2] for i in range(n)]
    Bs = [inputs[i][1] for i in range(n)] + [None] * n
    dep = [-1] * n + list(range(n))
    return As, Bs, dep, inputs
