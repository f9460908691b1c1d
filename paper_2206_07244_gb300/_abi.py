"""ctypes mirror of include/opsparse.h (argument marshalling only)."""

from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libopsparse.so")
MAX_BINS = 16

ERRORS = {0: "SPGEMM_OK", -1: "SPGEMM_ERR_INVALID", -2: "SPGEMM_ERR_SHAPE",
          -3: "SPGEMM_ERR_OOM", -4: "SPGEMM_ERR_STATE", -5: "SPGEMM_ERR_TIMEOUT",
          -6: "SPGEMM_ERR_CUDA", -7: "SPGEMM_ERR_INTERNAL", -8: "SPGEMM_ERR_ABORTED"}

# Every function the header declares (the CPU tests check the library
# exports them all).
EXPORTS = [
    "spgemm_create", "spgemm_set_config", "spgemm_get_config", "spgemm_symbolic",
    "spgemm_numeric", "spgemm_numeric_values", "spgemm_multiply", "spgemm_status", "spgemm_free",
    "spgemm_destroy", "spgemm_last_stats", "spgemm_kernel_info", "spgemm_strerror",
    "spgemm_last_cuda_error",
    "spgemm_multiply_host", "spgemm_bin_stats", "spgemm_window_stats", "spgemm_set_timing",
    "spgemm_kernel_times", "spgemm_set_phase_clocks", "spgemm_bitmap_phase_clocks",
    "spgemm_rowptr_noalloc", "spgemm_mlp_param_count", "spgemm_set_predictor", "spgemm_set_mode",
    "spgemm_learned_stats", "spgemm_features", "spgemm_mlp_forward", "spgemm_mlp_train_step",
    "spgemm_mlp_adam", "spgemm_batch_create", "spgemm_batch_run", "spgemm_batch_sync",
    "spgemm_batch_result", "spgemm_batch_info", "spgemm_batch_destroy", "spgemm_probe",
]


class SpgemmError(RuntimeError):
    def __init__(self, code: int, where: str, cuda: str | None = None):
        self.code = code
        self.cuda = cuda
        extra = f" ({cuda})" if cuda else ""
        super().__init__(f"{where}: {ERRORS.get(code, code)}{extra}")


class CsrIn(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rpt", ctypes.c_void_p), ("rpt_is_i64", ctypes.c_int32),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class CsrOut(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rpt", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class BatchOptions(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64), ("no_tiny", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Config(ctypes.Structure):
    _fields_ = [("sym_nbins", ctypes.c_int32), ("sym_kernel", ctypes.c_int32 * MAX_BINS),
                ("sym_range", ctypes.c_int64 * MAX_BINS),
                ("num_nbins", ctypes.c_int32), ("num_kernel", ctypes.c_int32 * MAX_BINS),
                ("num_range", ctypes.c_int64 * MAX_BINS),
                ("lanes_per_brow", ctypes.c_int32), ("num_lanes_per_brow", ctypes.c_int32),
                ("bitmap_unroll", ctypes.c_int32), ("window_lists", ctypes.c_int32),
                ("window_entries", ctypes.c_int32), ("hash_access", ctypes.c_int32),
                ("bitmap_path", ctypes.c_int32), ("window_budget", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
SINK_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64)

_lib = None
_lock = threading.Lock()


def lib(path: str | None = None):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"CUDA library not built: {p} is missing "
                              "(run paper_2206_07244_gb300.build())")
        L = ctypes.CDLL(p)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        sig = {
            "spgemm_create": [ctypes.POINTER(P), P, ALLOC_FN, FREE_FN, P, P],
            "spgemm_set_config": [P, P],
            "spgemm_get_config": [P, P],
            "spgemm_symbolic": [P, P, P, I64, I64, ctypes.POINTER(I64)],
            "spgemm_numeric": [P, P, P, P],
            "spgemm_numeric_values": [P, P, P, P],
            "spgemm_multiply": [P, P, P, P],
            "spgemm_status": [P],
            "spgemm_free": [P, P],
            "spgemm_destroy": [P],
            "spgemm_last_stats": [P, ctypes.POINTER(I64), ctypes.c_int],
            "spgemm_kernel_info": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(I32),
                                   ctypes.POINTER(I32), ctypes.POINTER(I64), ctypes.POINTER(I64)],
            "spgemm_multiply_host": [P, P, P, I64, SINK_FN, P, ctypes.POINTER(I64)],
            "spgemm_bin_stats": [P, ctypes.c_int, ctypes.POINTER(I64), ctypes.c_int],
            "spgemm_window_stats": [P, ctypes.POINTER(I64), ctypes.c_int],
            "spgemm_set_timing": [P, ctypes.c_int],
            "spgemm_rowptr_noalloc": [P, P, P, P, ctypes.POINTER(I64)],
            "spgemm_mlp_param_count": [],
            "spgemm_batch_create": [ctypes.POINTER(P), P, ctypes.c_int, P, P, P, P],
            "spgemm_batch_run": [P],
            "spgemm_batch_sync": [P],
            "spgemm_batch_result": [P, ctypes.c_int, P],
            "spgemm_batch_info": [P, ctypes.POINTER(I64), ctypes.c_int],
            "spgemm_batch_destroy": [P],
            "spgemm_probe": [ctypes.c_int, ctypes.c_int, I64, P, I64, ctypes.POINTER(ctypes.c_double), P],
            "spgemm_set_predictor": [P, P, ctypes.c_float],
            "spgemm_set_mode": [P, ctypes.c_int],
            "spgemm_learned_stats": [P, ctypes.POINTER(I64), ctypes.c_int],
            "spgemm_features": [P, P, I64, I64, P, P, P],
            "spgemm_mlp_forward": [P, P, I64, P, P],
            "spgemm_mlp_train_step": [P, P, P, I64, I64, P, P, P],
            "spgemm_mlp_adam": [P, P, P, P, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, ctypes.c_float, P],
            "spgemm_kernel_times": [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64),
                                    ctypes.c_int, ctypes.c_int],
            "spgemm_set_phase_clocks": [P, ctypes.c_int],
            "spgemm_bitmap_phase_clocks": [P, ctypes.POINTER(I64), ctypes.c_int, ctypes.c_int],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.spgemm_strerror.argtypes = [ctypes.c_int]
        L.spgemm_strerror.restype = ctypes.c_char_p
        L.spgemm_last_cuda_error.argtypes = []
        L.spgemm_last_cuda_error.restype = ctypes.c_char_p
        _lib = L
        return _lib


def check(rc: int, where: str):
    if rc != 0:
        cuda = None
        if rc in (-3, -6) and _lib is not None:
            name = _lib.spgemm_last_cuda_error()
            cuda = name.decode() if name else None
        raise SpgemmError(rc, where, cuda)


def kernel_table(phase: int):
    L = lib()
    out = []
    i = 0
    while True:
        tpr, blk = ctypes.c_int32(), ctypes.c_int32()
        tab, mx = ctypes.c_int64(), ctypes.c_int64()
        rc = L.spgemm_kernel_info(phase, i, ctypes.byref(tpr), ctypes.byref(blk),
                                  ctypes.byref(tab), ctypes.byref(mx))
        if rc != 0:
            return out
        out.append((tpr.value, blk.value, tab.value, mx.value))
        i += 1


def config_to_dict(c: Config) -> dict:
    return {"sym_kernel": list(c.sym_kernel[:c.sym_nbins]),
            "sym_range": list(c.sym_range[:c.sym_nbins]),
            "num_kernel": list(c.num_kernel[:c.num_nbins]),
            "num_range": list(c.num_range[:c.num_nbins]),
            "lanes_per_brow": int(c.lanes_per_brow),
            "num_lanes_per_brow": int(c.num_lanes_per_brow),
            "bitmap_unroll": int(c.bitmap_unroll),
            "window_lists": int(c.window_lists), "window_entries": int(c.window_entries),
            "hash_access": int(c.hash_access), "bitmap_path": int(c.bitmap_path),
            "window_budget": int(c.window_budget)}


def config_from_dict(d: dict) -> Config:
    c = Config()
    sk, sr = list(d["sym_kernel"]), list(d["sym_range"])
    nk, nr = list(d["num_kernel"]), list(d["num_range"])
    if len(sk) != len(sr) or len(nk) != len(nr) or not sk or not nk \
            or len(sk) > MAX_BINS or len(nk) > MAX_BINS:
        raise ValueError("bad bin configuration")
    c.sym_nbins, c.num_nbins = len(sk), len(nk)
    for j, (k, r) in enumerate(zip(sk, sr)):
        c.sym_kernel[j], c.sym_range[j] = int(k), int(r)
    for j, (k, r) in enumerate(zip(nk, nr)):
        c.num_kernel[j], c.num_range[j] = int(k), int(r)
    c.lanes_per_brow = int(d.get("lanes_per_brow", 0))
    c.num_lanes_per_brow = int(d.get("num_lanes_per_brow", 0))
    c.bitmap_unroll = int(d.get("bitmap_unroll", 0))
    c.window_lists = int(d.get("window_lists", 0))
    c.window_entries = int(d.get("window_entries", 0))
    c.hash_access = int(d.get("hash_access", 0))
    c.bitmap_path = int(d.get("bitmap_path", 0))
    c.window_budget = int(d.get("window_budget", 0))
    return c
