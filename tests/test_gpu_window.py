"""GPU parity of the numeric bitmap kernel's windowed pass 2 (B rows sorted:
values summed column window by column window over precomputed B-row runs)
against the CPU oracle, and of its fall-backs to the whole-row pass 2: rows
with more A entries than the windowed pass takes, B with unsorted rows, and
B wider than one bitmap. Small windows force many windows per row."""

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


def dev(m, rpt64=False):
    rpt = m.rpt.astype(np.int64) if rpt64 else m.rpt
    return ops.CSR.from_arrays(m.rows, m.cols, rpt, m.col, m.val)


def bitmap_only(window_lists=1024, window_entries=0):
    """Every numeric row to the bitmap kernel; symbolic defaults."""
    cfg = ops.default_config()
    bitmap = len(ops.kernel_table(1)) - 1
    cfg["num_kernel"], cfg["num_range"] = [bitmap], [-1]
    cfg.update(window_lists=window_lists, window_entries=window_entries)
    return cfg


def run(A, B, cfg, rpt64=False):
    with ops.Handle(cfg) as h:
        C = h.multiply(dev(A, rpt64), dev(B, rpt64))
        h.status()
        return C.numpy()


def check(A, B, got, exact=False):
    rpt, col, val, ab = oracle.spgemm(A, B)
    assert np.array_equal(got[0], rpt), "row pointers differ"
    assert np.array_equal(got[1], col), "column indices differ"
    if exact:
        assert np.array_equal(got[2], val)
    else:
        assert_values_close(got[2], val, ab)


@pytest.mark.parametrize("entries", [0, 64, 500, 3000])
def test_windowed_pass2_rmat(entries):
    A = W.rmat(12, 16, seed=21)
    check(A, A, run(A, A, bitmap_only(window_entries=entries)))


def test_windowed_pass2_integer_values_exact():
    A = W.random_csr(700, 900, 0.03, seed=5, integer_values=True)
    B = W.random_csr(900, 5000, 0.02, seed=6, integer_values=True)
    check(A, B, run(A, B, bitmap_only(window_entries=100)), exact=True)


def test_rows_split_between_windowed_and_whole_row():
    # rows with more than 20 A entries take the whole-row pass 2
    A = W.rmat(12, 16, seed=22)
    alen = np.diff(A.rpt.astype(np.int64))
    assert (alen > 20).any() and ((alen <= 20) & (alen > 0)).any()
    check(A, A, run(A, A, bitmap_only(window_lists=20, window_entries=256)))


def test_whole_row_pass2_alone():
    A = W.rmat(12, 16, seed=23)
    check(A, A, run(A, A, bitmap_only(window_lists=0)))


def test_every_row_whole_row():
    A = W.random_csr(64, 2000, 0.05, seed=7)     # about 100 A entries per row
    B = W.random_csr(2000, 3000, 0.01, seed=8)
    check(A, B, run(A, B, bitmap_only(window_lists=1)))


def test_unsorted_b_falls_back():
    A = W.random_csr(300, 400, 0.05, seed=9)
    B = W.random_csr(400, 2500, 0.02, seed=10, unsorted=True)
    check(A, B, run(A, B, bitmap_only(window_entries=64)))


def test_sorted_b_with_duplicate_columns():
    A = W.random_csr(300, 400, 0.05, seed=11, integer_values=True)
    B = W.random_csr(400, 2500, 0.02, seed=12, duplicates=True, integer_values=True)
    check(A, B, run(A, B, bitmap_only(window_entries=64)), exact=True)


def test_wide_b_one_bitmap():
    # 300,000 columns: one bitmap, 37 sub-ranges of 8,192 columns
    A = W.random_csr(48, 3000, 0.02, seed=13)
    B = W.random_csr(3000, 300_000, 0.0004, seed=14)
    check(A, B, run(A, B, bitmap_only(window_entries=1000)))


def test_b_wider_than_one_bitmap():
    # 2.5M columns: several bitmap windows per row, whole-row pass 2
    A = W.random_csr(16, 3000, 0.02, seed=18)
    B = W.random_csr(3000, 2_500_000, 0.00004, seed=19)
    check(A, B, run(A, B, bitmap_only()))


def test_dense_rows_many_windows():
    # rows of about 66,000 entries in 120,000 columns
    A = W.from_dense(np.ones((3, 40)))
    B = W.random_csr(40, 120_000, 0.02, seed=15)
    got = run(A, B, bitmap_only(window_entries=2000))
    check(A, B, got)
    assert np.diff(got[0]).max() > 40_000


def test_empty_rows_and_int64_pointers():
    A = W.random_csr(500, 300, 0.04, seed=16)
    A.rpt[100:200] = A.rpt[100]        # rows 100..198 empty, row 199 takes their entries
    B = W.random_csr(300, 4000, 0.03, seed=17)
    check(A, B, run(A, B, bitmap_only(window_entries=300), rpt64=True))


def test_default_config_rmat():
    A = W.rmat(13, 16, seed=24)
    check(A, A, run(A, A, None))


def test_window_options_validated():
    cfg = bitmap_only(window_lists=1025)
    with pytest.raises(ops.SpgemmError):
        ops.Handle(cfg)
