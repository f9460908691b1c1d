"""GPU parity of the column-window forms of the large rows (the last numeric
bin).

bitmap_path 1: one block per row, two per SM, each row covered in column
windows of half an SM's shared memory that walk only the runs of sorted B
rows inside them. bitmap_path 2 (window.cu): rows cut into windows
planned from per-cell counts and summed in shared memory, by column where a
window is dense, by rank in a column bitmap elsewhere, one window over all
columns for small rows.
Every case is compared with the CPU oracle element by element (structure bit
for bit, values within helpers.VALUE_RTOL, integer-valued inputs bit for
bit), and window_stats() shows which kind of window ran, so each form is
checked on purpose rather than by accident of the input."""

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


def windows_only(budget=0, path=2):
    """Every row to the symbolic and numeric bitmap bins (so every row has
    cell counts and every row of C goes through the window kernel)."""
    cfg = ops.default_config()
    sb = len(ops.kernel_table(0)) - 1
    nb = len(ops.kernel_table(1)) - 1
    cfg["sym_kernel"], cfg["sym_range"] = [sb], [-1]
    cfg["num_kernel"], cfg["num_range"] = [nb], [-1]
    cfg["bitmap_path"] = path
    cfg["window_budget"] = budget
    return cfg


def dev(m):
    return ops.CSR.from_arrays(m.rows, m.cols, m.rpt, m.col, m.val)


def run(A, B, cfg=None, r0=0, r1=None):
    with ops.Handle(cfg) as h:
        dA, dB = dev(A), dev(B)
        h.symbolic(dA, dB, r0, A.rows if r1 is None else r1)
        C = h.numeric(dA, dB)
        h.status()
        return C.numpy(), h.window_stats()


def check(A, B, got, exact=False, r0=0, r1=None):
    rpt, col, val, ab = oracle.spgemm(A, B, r0, r1)
    g_rpt, g_col, g_val = got
    assert np.array_equal(g_rpt, rpt), "row pointers differ"
    assert np.array_equal(g_col, col), "column indices differ"
    if exact:
        assert np.array_equal(g_val, val), "values differ (exact case)"
    else:
        assert_values_close(g_val, val, ab)


def wide_dense(rows, k, ncols, per_row, span, seed, dup=False):
    """A (rows x k, every row referencing all k rows of B) times B (k x ncols)
    whose rows hold per_row sorted columns drawn from [0, span): products that
    pile up on the same columns, so C's rows are dense inside [0, span)."""
    rng = np.random.default_rng(seed)
    ar = np.repeat(np.arange(rows), k)
    ac = np.tile(np.arange(k), rows)
    av = rng.uniform(-1, 1, ar.size)
    A = W._from_coo(rows, k, ar, ac, av)
    br, bc = [], []
    for i in range(k):
        c = np.sort(rng.choice(span, per_row, replace=False))
        if dup and i % 3 == 0:
            c = np.sort(np.concatenate([c, c[: per_row // 4]]))   # equal columns inside a row
        br.append(np.full(c.size, i))
        bc.append(c)
    br = np.concatenate(br)
    bc = np.concatenate(bc)
    B = W.Csr(k, ncols, np.concatenate([[0], np.cumsum(np.bincount(br, minlength=k))]).astype(np.int64),
              bc.astype(np.int32), rng.uniform(-1, 1, bc.size))
    return A, B


def test_whole_width_windows_rmat14():
    A = W.rmat(14, 8, seed=5)
    got, st = run(A, A, windows_only())
    assert st["used"] and st["column_windows"] == 0
    assert st["windows"] == int(np.count_nonzero(oracle.symbolic(A, A)))
    check(A, A, got)


def test_small_budget_rank_and_column_windows_rmat18():
    # a 40000-byte window holds a bitmap of 213K columns: no row of a 2^18-column
    # product fits one window, so every row is planned from its cell counts,
    # into column windows (dense cells) and rank windows (the rest)
    A = W.rmat(18, 8, seed=7)
    got, st = run(A, A, windows_only(budget=40000), 0, 4096)
    assert st["used"] and st["whole_width_max"] == -1 and st["column_windows"] > 0
    nz = int(np.count_nonzero(oracle.symbolic(A, A, 0, 4096)))
    assert st["windows"] > st["column_windows"] and st["windows"] > nz
    check(A, A, got, r0=0, r1=4096)


def test_dense_rows_take_column_windows():
    A, B = wide_dense(48, 64, 1 << 20, 3000, 1 << 17, seed=11)
    got, st = run(A, B, windows_only())
    assert st["used"] and st["column_windows"] > 0
    check(A, B, got)


def test_duplicate_columns_in_rows_of_a_and_b():
    A, B = wide_dense(24, 48, 1 << 19, 2500, 1 << 16, seed=12, dup=True)
    ar, ac, av = [], [], []
    for i in range(A.rows):   # every A row references B row 0 twice more
        ar += [i, i]
        ac += [0, 0]
        av += [0.5, -0.25]
    A2 = W._from_coo(A.rows, A.cols,
                     np.concatenate([np.repeat(np.arange(A.rows), np.diff(A.rpt)), ar]),
                     np.concatenate([A.col, ac]), np.concatenate([A.val, av]), merge=False)
    got, st = run(A2, B, windows_only(budget=60000))
    assert st["used"]
    check(A2, B, got)


def test_integer_values_exact_laplacian():
    A = W.laplacian_2d(64)
    got, st = run(A, A, windows_only(budget=40000))
    assert st["used"]
    check(A, A, got, exact=True)


def test_row_window_of_heavy_rmat18_rows():
    A = W.rmat(18, 16, seed=9)
    got, st = run(A, A, windows_only(), 0, 3000)
    assert st["used"] and st["windows"] > 0
    check(A, A, got, r0=0, r1=3000)


def test_cells_across_symbolic_passes():
    # 3M columns: the symbolic bitmap kernel covers them in two passes, the
    # cells of both passes must add up
    A, B = wide_dense(8, 32, 3_000_000, 20000, 3_000_000, seed=13)
    got, st = run(A, B, windows_only())
    assert st["used"] and st["cells"] == -(-3_000_000 // (1 << st["cell_log2"]))
    check(A, B, got)


def test_unsorted_b_keeps_whole_row_kernel():
    A, B = wide_dense(16, 32, 1 << 18, 2000, 1 << 16, seed=14)
    col = B.col.copy()
    col[B.rpt[3]:B.rpt[4]] = col[B.rpt[3]:B.rpt[4]][::-1]   # one row of B decreasing
    B2 = W.Csr(B.rows, B.cols, B.rpt, col, B.val.copy())
    got, st = run(A, B2, windows_only())
    assert st["planned"] and not st["used"]
    check(A, B2, got)


def test_wide_b_keeps_whole_row_kernel():
    A, B = wide_dense(4, 8, 1 << 23, 500, 1 << 23, seed=15)
    got, st = run(A, B, windows_only())
    assert not st["planned"]
    check(A, B, got)


def test_forced_whole_row_kernel_matches():
    A = W.rmat(15, 16, seed=16)
    got, st = run(A, A, windows_only(path=0))
    assert not st["used"]
    check(A, A, got)


def test_numeric_values_reuses_windows():
    A = W.rmat(18, 8, seed=17)
    with ops.Handle(windows_only(budget=40000)) as h:
        dA = dev(A)
        h.symbolic(dA, dA, 0, 4096)
        C = h.numeric(dA, dA)
        st = h.window_stats()
        assert st["used"] and st["column_windows"] > 0
        rng = np.random.default_rng(3)
        for _ in range(2):
            A2 = W.Csr(A.rows, A.cols, A.rpt, A.col, rng.uniform(-2, 2, A.nnz))
            C2 = h.numeric_values(dev(A2), dev(A2), C)
            h.status()
            check(A2, A2, C2.numpy(), r0=0, r1=4096)


# --- the default form: run-restricted half-width windows, two blocks per SM ---

def bitmap_bin_only(path=1):
    """Every row of C to the numeric bitmap kernel, default symbolic bins."""
    cfg = ops.default_config()
    nb = len(ops.kernel_table(1)) - 1
    cfg["num_kernel"], cfg["num_range"] = [nb], [-1]
    cfg["bitmap_path"] = path
    return cfg


def test_split_windows_wide_rows():
    # 2^20 columns: two windows per row, the second found through the index
    A, B = wide_dense(48, 64, 1 << 20, 3000, 1 << 20, seed=21)
    got, st = run(A, B, bitmap_bin_only())
    assert st["split"]
    check(A, B, got)


def test_split_windows_many_windows_and_duplicates():
    # 3M columns: six windows per row; B rows with repeated columns
    A, B = wide_dense(12, 40, 3_000_000, 8000, 3_000_000, seed=22, dup=True)
    got, st = run(A, B, bitmap_bin_only())
    assert st["split"]
    check(A, B, got)


def test_split_single_window_rmat16_every_row():
    A = W.rmat(16, 16, seed=23)
    got, st = run(A, A, bitmap_bin_only())
    assert st["split"]
    check(A, A, got)


def test_split_integer_values_exact():
    A = W.laplacian_2d(64)
    got, st = run(A, A, bitmap_bin_only())
    assert st["split"]
    check(A, A, got, exact=True)


def test_split_unsorted_b_takes_whole_width():
    A, B = wide_dense(16, 32, 1 << 20, 2000, 1 << 20, seed=24)
    col = B.col.copy()
    col[B.rpt[5]:B.rpt[6]] = col[B.rpt[5]:B.rpt[6]][::-1]
    B2 = W.Csr(B.rows, B.cols, B.rpt, col, B.val.copy())
    got, st = run(A, B2, bitmap_bin_only())
    assert not st["split"]
    check(A, B2, got)


def test_default_path_is_whole_width():
    A, B = wide_dense(16, 32, 1 << 20, 2000, 1 << 20, seed=25)
    got, st = run(A, B, bitmap_bin_only(path=0))
    assert not st["split"]
    check(A, B, got)


def test_split_numeric_values_rerun():
    A, B = wide_dense(24, 48, 1 << 20, 2500, 1 << 20, seed=26)
    with ops.Handle(bitmap_bin_only()) as h:
        dA, dB = dev(A), dev(B)
        C = h.multiply(dA, dB)
        assert h.window_stats()["split"]
        rng = np.random.default_rng(5)
        for _ in range(2):
            B2 = W.Csr(B.rows, B.cols, B.rpt, B.col, rng.uniform(-2, 2, B.nnz))
            C2 = h.numeric_values(dA, dev(B2), C)
            h.status()
            check(A, B2, C2.numpy())


def test_default_form_walks_runs_when_columns_exceed_one_bitmap():
    # 3M columns do not fit one bitmap: the default form covers each row in
    # windows that walk only their runs (sorted B)
    A, B = wide_dense(10, 40, 3_000_000, 9000, 3_000_000, seed=27)
    got, st = run(A, B, bitmap_bin_only(path=0))
    assert st["split"]
    check(A, B, got)


def test_default_form_unsorted_wide_b():
    # the symbolic bitmap kernel's runs are switched off on the device when
    # some row of B is unsorted; the numeric kernel walks whole rows
    A, B = wide_dense(8, 30, 3_000_000, 9000, 3_000_000, seed=28)
    col = B.col.copy()
    col[B.rpt[2]:B.rpt[3]] = col[B.rpt[2]:B.rpt[3]][::-1]
    B2 = W.Csr(B.rows, B.cols, B.rpt, col, B.val.copy())
    got, st = run(A, B2)
    assert not st["split"]
    check(A, B2, got)


def test_learned_mode_wide_b_exact_rows_walk_runs():
    from paper_2206_07244_gb300 import learned
    A, B = wide_dense(10, 36, 3_000_000, 9000, 3_000_000, seed=29)
    theta = np.load(learned.WEIGHTS)
    with ops.Handle() as h:
        h.set_predictor(theta, 0.0)
        h.set_mode("learned")
        dA, dB = dev(A), dev(B)
        C = h.multiply(dA, dB)
        h.status()
        check(A, B, C.numpy())
