"""Pins for the CPU oracle: each test checks it against something other than
itself (closed forms, library dense products, brute force, the paper's own
tables), so that a dropped term, a wrong index or a transposed operand in the
oracle fails here. CPU only."""

import itertools

import numpy as np
import pytest

import oracle
import workloads as W
from helpers import assert_values_close, load_binning_golden


def oracle_dense(A, B):
    rpt, col, val, _ = oracle.spgemm(A, B)
    d = np.zeros((A.rows, B.cols))
    pattern = np.zeros((A.rows, B.cols), dtype=bool)
    for i in range(A.rows):
        for p in range(rpt[i], rpt[i + 1]):
            assert not pattern[i, col[p]], "duplicate column in an output row"
            d[i, col[p]] = val[p]
            pattern[i, col[p]] = True
    return d, pattern, rpt, col, val


def test_tridiagonal_square_closed_form():
    # T = tridiag(-1, 2, -1): T^2 has rows [5,-4,1], [-4,6,-4,1],
    # [1,-4,6,-4,1] (interior), mirrored at the end; nnz = 5n - 6.
    for n in (5, 6, 11, 64):
        T = W.tridiag_1d(n)
        rpt, col, val, _ = oracle.spgemm(T, T)
        assert rpt[-1] == 5 * n - 6
        rows = {i: (list(col[rpt[i]:rpt[i + 1]]), list(val[rpt[i]:rpt[i + 1]]))
                for i in range(n)}
        assert rows[0] == ([0, 1, 2], [5.0, -4.0, 1.0])
        assert rows[1] == ([0, 1, 2, 3], [-4.0, 6.0, -4.0, 1.0])
        assert rows[n - 1] == ([n - 3, n - 2, n - 1], [1.0, -4.0, 5.0])
        assert rows[n - 2] == ([n - 4, n - 3, n - 2, n - 1], [1.0, -4.0, 6.0, -4.0])
        for i in range(2, n - 2):
            assert rows[i] == ([i - 2, i - 1, i, i + 1, i + 2],
                               [1.0, -4.0, 6.0, -4.0, 1.0])


@pytest.mark.parametrize("seed", range(6))
def test_against_dense_product(seed):
    # Rectangular shapes (M != K != N) catch a transposed operand.
    rng = np.random.default_rng(100 + seed)
    m, k, n = rng.integers(1, 17, size=3)
    dens = [0.05, 0.2, 0.5, 1.0][seed % 4]
    A = W.random_csr(int(m), int(k), dens, seed=seed, duplicates=seed % 2 == 1,
                     unsorted=seed % 3 == 2)
    B = W.random_csr(int(k), int(n), dens, seed=50 + seed, duplicates=seed % 3 == 1,
                     unsorted=seed % 2 == 0)
    d, pattern, rpt, col, val = oracle_dense(A, B)
    Ad, Bd = A.to_dense(), B.to_dense()
    want = Ad @ Bd
    # structure: (i, j) is stored iff some stored A(i,k) meets a stored B(k,j)
    Ap = np.zeros((A.rows, A.cols), dtype=np.int64)
    Bp = np.zeros((B.rows, B.cols), dtype=np.int64)
    for i in range(A.rows):
        Ap[i, A.col[A.rpt[i]:A.rpt[i + 1]]] = 1
    for i in range(B.rows):
        Bp[i, B.col[B.rpt[i]:B.rpt[i + 1]]] = 1
    assert np.array_equal(pattern, (Ap @ Bp) > 0)
    scale = np.abs(Ad) @ np.abs(Bd)
    assert_values_close(d[pattern], want[pattern], scale[pattern])
    assert np.all(want[~pattern] == 0.0)
    # every output row sorted ascending
    for i in range(A.rows):
        assert np.all(np.diff(col[rpt[i]:rpt[i + 1]]) > 0)


def brute_force(A, B):
    """Triple loop over stored entries, pure Python, dict accumulator."""
    out = []
    for i in range(A.rows):
        acc = {}
        for p in range(int(A.rpt[i]), int(A.rpt[i + 1])):
            k = int(A.col[p])
            for q in range(int(B.rpt[k]), int(B.rpt[k + 1])):
                j = int(B.col[q])
                acc[j] = acc.get(j, 0.0) + float(A.val[p]) * float(B.val[q])
        out.append(sorted(acc.items()))
    return out


@pytest.mark.parametrize("seed", range(4))
def test_brute_force_integer_values_bit_exact(seed):
    A = W.random_csr(40 + seed, 30, 0.15, seed=seed, duplicates=True,
                     unsorted=True, integer_values=True)
    B = W.random_csr(30, 64 - seed, 0.2, seed=10 + seed, duplicates=True,
                     integer_values=True)
    want = brute_force(A, B)
    rpt, col, val, _ = oracle.spgemm(A, B)
    for i, row in enumerate(want):
        got = list(zip(col[rpt[i]:rpt[i + 1]].tolist(), val[rpt[i]:rpt[i + 1]].tolist()))
        assert got == row, i


def test_identity_products_are_exact():
    A = W.random_csr(33, 21, 0.3, seed=7)
    for left, right in ((W.identity(33), A), (A, W.identity(21))):
        rpt, col, val, _ = oracle.spgemm(left, right)
        assert np.array_equal(rpt, A.rpt.astype(np.int64))
        assert np.array_equal(col, A.col)
        assert np.array_equal(val, A.val)


def test_permutation_products():
    rng = np.random.default_rng(3)
    A = W.random_csr(25, 25, 0.25, seed=9)
    perm = rng.permutation(25)
    P = W.permutation(perm)
    Ad = A.to_dense()
    # (P A)(i, :) = A(perm[i], :)
    d, _, _, _, _ = oracle_dense(P, A)
    assert np.array_equal(d, Ad[perm, :])
    # (A P)(:, perm[k]) = A(:, k)
    d, _, _, _, _ = oracle_dense(A, P)
    want = np.zeros_like(Ad)
    want[:, perm] = Ad
    assert np.array_equal(d, want)


def test_zero_and_empty_operands():
    A = W.random_csr(10, 8, 0.3, seed=1)
    Z = W.Csr(8, 12, np.zeros(9, dtype=np.int32), np.zeros(0, dtype=np.int32),
              np.zeros(0))
    rpt, col, val, _ = oracle.spgemm(A, Z)
    assert rpt.shape == (11,) and rpt[-1] == 0 and col.size == 0
    E = W.Csr(0, 8, np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    rpt, col, val, _ = oracle.spgemm(E, W.random_csr(8, 5, 0.5, seed=2))
    assert rpt.tolist() == [0]


def test_cancellation_keeps_structural_entry():
    # Row [1, 1] times rows [1] and [-1] at the same column: the sum is 0.0
    # but the symbolic phase counts the key, so the entry stays.
    A = W.Csr(1, 2, np.array([0, 2], dtype=np.int32), np.array([0, 1], dtype=np.int32),
              np.array([1.0, 1.0]))
    B = W.Csr(2, 3, np.array([0, 1, 2], dtype=np.int32), np.array([2, 2], dtype=np.int32),
              np.array([1.0, -1.0]))
    rpt, col, val, _ = oracle.spgemm(A, B)
    assert rpt.tolist() == [0, 1] and col.tolist() == [2] and val.tolist() == [0.0]


def test_laplacian_2d_kronecker_identity():
    # A = I (x) T + T (x) I, so A^2 = I (x) T^2 + 2 T (x) T + T^2 (x) I
    # (all entries small integers: exact in float64).
    nx, ny = 6, 5
    A = W.laplacian_2d(nx, ny)
    Tx = W.tridiag_1d(nx).to_dense()
    Ty = W.tridiag_1d(ny).to_dense()
    want = (np.kron(np.eye(ny), Tx @ Tx) + 2 * np.kron(Ty, Tx)
            + np.kron(Ty @ Ty, np.eye(nx)))
    d, pattern, _, _, _ = oracle_dense(A, A)
    assert np.array_equal(d, want)
    # structure: the 13-point diamond |dx| + |dy| <= 2 clipped to the grid
    for i, j in itertools.product(range(nx * ny), repeat=2):
        dx = abs(i % nx - j % nx)
        dy = abs(i // nx - j // nx)
        assert pattern[i, j] == (dx + dy <= 2)


def test_laplacian_2d_64_statistics():
    # 64x64 grid: corner rows have 3 entries, other edge rows 4, interior 5.
    # A is symmetric, so total n_prod = sum over rows k of len_k^2.
    A = W.laplacian_2d(64)
    nprod = oracle.nprod(A, A)
    assert nprod.sum() == 4 * 9 + 4 * 62 * 16 + 62 * 62 * 25 == 100104
    nnz = oracle.symbolic(A, A)
    # clipped 13-point diamond, counted point by point
    total = 0
    for x in range(64):
        for y in range(64):
            for dx in range(-2, 3):
                for dy in range(-2, 3):
                    if abs(dx) + abs(dy) <= 2 and 0 <= x + dx < 64 and 0 <= y + dy < 64:
                        total += 1
    assert nnz.sum() == total == 51972
    assert nnz.max() == 13


@pytest.mark.parametrize("s", [3, 5, 6])
def test_stencil27_structure_closed_form(s):
    # The 27-point pattern is (tridiagonal pattern)^(x)3, so C's pattern is
    # (pentadiagonal pattern)^(x)3: nnz(C) = (5s - 6)^3; and n_prod =
    # (sum_k len_k^2)^3 with 1D lengths 2, 3, ..., 3, 2: (9s - 10)^3.
    A = W.stencil27(s, seed=3)
    assert A.nnz == (3 * s - 2) ** 3
    assert oracle.nprod(A, A).sum() == (9 * s - 10) ** 3
    assert oracle.symbolic(A, A).sum() == (5 * s - 6) ** 3


@pytest.mark.parametrize("s", [4, 6, 8])
def test_galerkin_even_side_identity(s):
    # For even s, P^T (A P) with 2x2x2 aggregation of the 7-point Dirichlet
    # Laplacian is 4 * L7(s/2): each aggregate has 8 points with diagonal 6
    # and 12 internal edges (8*6 - 2*12 = 24), and 4 edges cross each
    # coarse face (-4).
    A, P, PT = W.galerkin_problem(s)
    AP = oracle.spgemm_csr(A, P)
    assert AP.rpt[-1] > 0
    Ac = oracle.spgemm_csr(PT, AP)
    L = W.laplacian_3d_7pt(s // 2)
    assert np.array_equal(Ac.rpt, L.rpt.astype(np.int64))
    assert np.array_equal(Ac.col, L.col)
    assert np.array_equal(Ac.val, 4.0 * L.val)
    # n_prod(A P) = nnz(A): every row of P has exactly one entry
    assert oracle.nprod(A, P).sum() == A.nnz


def test_nprod_hand_example():
    # A rows: {0, 2}, {}, {1, 1(dup)}, B row lengths 3, 1, 2.
    A = W.Csr(3, 3, np.array([0, 2, 2, 4], dtype=np.int32),
              np.array([0, 2, 1, 1], dtype=np.int32), np.ones(4))
    B = W.Csr(3, 4, np.array([0, 3, 4, 6], dtype=np.int32),
              np.array([0, 1, 3, 2, 0, 3], dtype=np.int32), np.ones(6))
    assert oracle.nprod(A, B).tolist() == [5, 0, 2]
    assert oracle.symbolic(A, B).tolist() == [3, 0, 1]


@pytest.mark.parametrize("seed", range(3))
def test_count_invariants(seed):
    A = W.random_csr(200, 150, 0.05, seed=seed, duplicates=True)
    B = W.random_csr(150, 120, 0.08, seed=seed + 5)
    nprod = oracle.nprod(A, B)
    nnz = oracle.symbolic(A, B)
    # sum_i n_prod(i) = sum_k (entries of A in column k) * (length of B row k)
    colcount = np.bincount(A.col, minlength=A.cols)
    assert nprod.sum() == int((colcount * np.diff(B.rpt.astype(np.int64))).sum())
    assert np.all(nnz <= np.minimum(nprod, B.cols))
    assert oracle.compression_ratio(nprod.sum(), nnz.sum()) >= 1.0
    rpt, _, _, _ = oracle.spgemm(A, B)
    assert np.array_equal(np.diff(rpt), nnz)


def test_row_checksums_agree_with_full_product():
    A = W.rmat(9, 8, seed=4)
    rpt, col, val, ab = oracle.spgemm(A, A)
    cnt, cs, vs, rab = oracle.row_checksums(A, A)
    assert np.array_equal(cnt, np.diff(rpt))
    for i in range(A.rows):
        assert cs[i] == int(col[rpt[i]:rpt[i + 1]].astype(np.int64).sum())
        acc = 0.0   # plain left-to-right sum (Python's sum() is compensated)
        for x in val[rpt[i]:rpt[i + 1]].tolist():
            acc += x
        assert vs[i] == acc
    # windowed calls see the same rows
    cnt2, cs2, vs2, rab2 = oracle.row_checksums(A, A, 100, 300)
    assert np.array_equal(cnt2, cnt[100:300]) and np.array_equal(vs2, vs[100:300])
    assert np.array_equal(rab2, rab[100:300])


def test_row_abs_sums_brute_force():
    """A row's sum of |a*b| over its intermediate products (the tolerance
    scale of its entries, Eq. 2's products), against a plain Python loop over
    A's and B's entries, and against the per-entry sums of the full product."""
    A = W.rmat(8, 6, seed=11)
    B = W.random_csr(A.cols, 40, 0.1, seed=12)
    rpt, col, val, ab = oracle.spgemm(A, B)
    _, _, _, rab = oracle.row_checksums(A, B)
    arpt, brpt = A.rpt.astype(np.int64), B.rpt.astype(np.int64)
    for i in range(A.rows):
        want = 0.0
        for p in range(arpt[i], arpt[i + 1]):
            k, a = int(A.col[p]), float(A.val[p])
            for q in range(brpt[k], brpt[k + 1]):
                want += abs(a * float(B.val[q]))
        assert rab[i] == pytest.approx(want, rel=1e-14, abs=0.0)
        assert rab[i] == pytest.approx(float(ab[rpt[i]:rpt[i + 1]].sum()), rel=1e-13, abs=0.0)


def test_row_window_matches_full():
    A = W.rmat(10, 8, seed=5)
    full = oracle.spgemm(A, A)
    r0, r1 = 123, 777
    rpt, col, val, _ = oracle.spgemm(A, A, r0, r1)
    s, e = full[0][r0], full[0][r1]
    assert np.array_equal(rpt, full[0][r0:r1 + 1] - s)
    assert np.array_equal(col, full[1][s:e]) and np.array_equal(val, full[2][s:e])


def test_binning_matches_paper_tables():
    ranges, cases = load_binning_golden()
    for table, size, want in cases:
        b = oracle.binning(np.array([size]), ranges[table])
        assert int(b["bin_of"][0]) == want, (table, size)


def test_binning_arrays():
    ranges, _ = load_binning_golden()
    sizes = np.array([5, 500, 0, 20000, 27, 26, 900, 5])
    b = oracle.binning(sizes, ranges["table1"])
    assert b["bin_size"].tolist() == [4, 1, 1, 1, 0, 0, 0, 1]
    assert b["bin_offset"].tolist() == [0, 4, 5, 6, 7, 7, 7, 7]
    assert b["bins"].tolist() == [0, 2, 5, 7, 4, 1, 6, 3]
    assert b["max"] == 20000
    assert sorted(b["bins"].tolist()) == list(range(sizes.size))


def test_exclusive_scan():
    assert oracle.exclusive_scan(np.array([3, 0, 2, 5])).tolist() == [0, 3, 3, 5, 10]
    assert oracle.exclusive_scan(np.array([], dtype=np.int64)).tolist() == [0]
    big = np.full(10000, 7, dtype=np.int64)
    out = oracle.exclusive_scan(big)
    assert out[-1] == 70000 and out[5000] == 35000


def test_bad_input_is_rejected():
    A = W.Csr(2, 3, np.array([0, 1, 2], dtype=np.int32), np.array([0, 3], dtype=np.int32),
              np.ones(2))
    with pytest.raises(ValueError):
        oracle.symbolic(A, W.identity(3))
    with pytest.raises(ValueError):
        oracle.nprod(A, W.identity(3))
    with pytest.raises(ValueError):
        oracle.nprod(W.identity(2), W.identity(3))
