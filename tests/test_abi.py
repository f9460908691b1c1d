"""The CUDA library builds for sm_103a, loads without a GPU, and exports
every function that include/opsparse.h declares. CPU only: no kernel runs."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    import paper_2206_07244_gb300 as ops
    return ops.build()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(spgemm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("spgemm_create", "spgemm_symbolic", "spgemm_numeric", "spgemm_destroy"):
        assert must in names


def test_library_exports_every_declared_function(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_python_binding_lists_the_same_functions():
    from paper_2206_07244_gb300 import _abi
    assert set(_abi.EXPORTS) == declared_functions()


def test_library_loads_and_answers_host_queries(libpath):
    from paper_2206_07244_gb300 import _abi
    L = _abi.lib(libpath)
    assert L.spgemm_strerror(0) == b"ok"
    assert L.spgemm_strerror(-2).startswith(b"shape")
    sym = _abi.kernel_table(0)
    num = _abi.kernel_table(1)
    assert len(sym) >= 8 and len(num) >= 8
    # the last kernel of each phase takes rows of any size (the bitmap)
    assert sym[-1][3] == -1 and num[-1][3] == -1
    # hash kernels: capacity grows with the bin
    assert all(a[3] < b[3] for a, b in zip(sym[:-2], sym[1:-1]))
    assert all(a[3] < b[3] for a, b in zip(num[:-2], num[1:-1]))
    # a numeric table can sort its rows in place: max size is a power of two <= table
    for tpr, blk, tab, mx in num[:-1]:
        assert mx <= tab and (mx & (mx - 1)) == 0
        assert blk % tpr == 0 or tpr == blk


def test_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2206_07244_gb300 import _abi
    L = _abi.lib(libpath)
    h = ctypes.c_void_p()
    rc = L.spgemm_create(ctypes.byref(h), None, _abi.ALLOC_FN(), _abi.FREE_FN(), None, None)
    assert rc == -6 and not h.value  # SPGEMM_ERR_CUDA, no handle


def test_config_dict_roundtrip():
    from paper_2206_07244_gb300 import _abi
    d = {"sym_kernel": [0, 9], "sym_range": [53, -1], "num_kernel": [2, 9],
         "num_range": [128, -1], "lanes_per_brow": 8, "num_lanes_per_brow": 32, "bitmap_unroll": 8,
         "window_lists": 300, "window_entries": 4096, "hash_access": 1, "bitmap_path": 1,
         "window_budget": 65536}
    assert _abi.config_to_dict(_abi.config_from_dict(d)) == d
    with pytest.raises(ValueError):
        _abi.config_from_dict({"sym_kernel": [0], "sym_range": [], "num_kernel": [1],
                               "num_range": [-1]})
