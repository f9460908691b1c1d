"""GPU parity: the CUDA path against the CPU oracle, element by element.

Structure (C.rpt, C.col) must match bit for bit; values within the
float64 summation bound of helpers.VALUE_RTOL, or bit for bit where every
partial sum is an exact integer. Every kernel of both phases is forced on
its own through the bin configuration, so each one is checked, not only the
bins a matrix happens to fill."""

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


@pytest.fixture(scope="module")
def handle():
    h = ops.Handle()
    yield h
    h.status()
    h.close()


def to_dev(m, rpt64=False):
    rpt = m.rpt.astype(np.int64) if rpt64 else m.rpt
    return ops.CSR.from_arrays(m.rows, m.cols, rpt, m.col, m.val)


def gpu_product(A, B, handle, rpt64=False):
    C = handle.multiply(to_dev(A, rpt64), to_dev(B, rpt64))
    handle.status()
    return C.numpy()


def check(A, B, got, exact=False, r0=0, r1=None):
    rpt, col, val, ab = oracle.spgemm(A, B, r0, r1)
    g_rpt, g_col, g_val = got
    assert g_rpt.dtype == np.int64
    assert np.array_equal(g_rpt, rpt), "row pointers differ"
    assert np.array_equal(g_col, col), "column indices differ"
    if exact:
        assert np.array_equal(g_val, val), "values differ (exact case)"
    else:
        assert_values_close(g_val, val, ab)


def forced(phase, kernel, lanes=0):
    """A configuration that sends every row it can to one kernel."""
    cfg = ops.default_config()
    table = ops.kernel_table(phase)
    key = "sym" if phase == 0 else "num"
    bitmap = len(table) - 1
    if kernel == bitmap:
        cfg[f"{key}_kernel"], cfg[f"{key}_range"] = [bitmap], [-1]
    else:
        cfg[f"{key}_kernel"] = [kernel, bitmap]
        cfg[f"{key}_range"] = [table[kernel][3], -1]
    cfg["lanes_per_brow"] = lanes
    return cfg


def test_laplacian_2d_64_bit_exact(handle):
    A = W.laplacian_2d(64)
    got = gpu_product(A, A, handle)
    check(A, A, got, exact=True)
    st = handle.stats()
    assert st["total_nprod"] == 100104 and st["total_nnz"] == 51972 and st["max_nnz"] == 13


def test_tridiagonal_square_gpu(handle):
    n = 5000
    T = W.tridiag_1d(n)
    rpt, col, val = gpu_product(T, T, handle)
    assert rpt[-1] == 5 * n - 6
    i = 2500
    assert col[rpt[i]:rpt[i + 1]].tolist() == [i - 2, i - 1, i, i + 1, i + 2]
    assert val[rpt[i]:rpt[i + 1]].tolist() == [1.0, -4.0, 6.0, -4.0, 1.0]


@pytest.mark.parametrize("seed", range(4))
def test_random_rectangular_integer_values(handle, seed):
    A = W.random_csr(300 + 17 * seed, 211, 0.04 * (seed + 1), seed=seed, duplicates=True,
                     unsorted=True, integer_values=True)
    B = W.random_csr(211, 333 - seed, 0.05, seed=40 + seed, duplicates=seed % 2 == 0,
                     unsorted=True, integer_values=True)
    check(A, B, gpu_product(A, B, handle), exact=True)


@pytest.mark.parametrize("scale,degree", [(10, 8), (12, 16)])
def test_rmat(handle, scale, degree):
    A = W.rmat(scale, degree, seed=11)
    check(A, A, gpu_product(A, A, handle))


def test_stencil27_structure_and_values(handle):
    s = 14
    A = W.stencil27(s, seed=3)
    got = gpu_product(A, A, handle)
    assert got[0][-1] == (5 * s - 6) ** 3
    assert handle.stats()["total_nprod"] == (9 * s - 10) ** 3
    check(A, A, got)


def test_int64_row_pointers(handle):
    A = W.rmat(11, 8, seed=2)
    check(A, A, gpu_product(A, A, handle, rpt64=True))


@pytest.mark.parametrize("kernel", range(len(ops.kernel_table(0)) if torch.cuda.is_available() else 0))
def test_each_symbolic_kernel(kernel):
    A = W.rmat(11, 12, seed=5)
    with ops.Handle(forced(0, kernel)) as h:
        got = gpu_product(A, A, h)
        bins = h.stats()["sym_bins"]
    check(A, A, got)
    assert bins[0] > 0  # the forced kernel did receive rows


@pytest.mark.parametrize("kernel", range(len(ops.kernel_table(1)) if torch.cuda.is_available() else 0))
def test_each_numeric_kernel(kernel):
    A = W.rmat(11, 12, seed=6)
    with ops.Handle(forced(1, kernel)) as h:
        got = gpu_product(A, A, h)
        bins = h.stats()["num_bins"]
    check(A, A, got)
    assert bins[0] > 0


def contended_product(seed):
    """Rows whose products pile onto a few columns: each A row has 100 to 250
    entries and every B row holds 6 to 10 of the same 12 columns, so many
    lanes update one table slot at once. Small integer values keep every
    sum exact in float64."""
    rng = np.random.default_rng(seed)
    m, k, n = 192, 300, 40
    a_rows = [np.sort(rng.choice(k, rng.integers(100, 251), replace=False)) for _ in range(m)]
    hot = rng.choice(n, 12, replace=False)
    b_rows = [np.sort(rng.choice(hot, rng.integers(6, 11), replace=False)) for _ in range(k)]

    def csr(rows, ncols):
        rpt = np.zeros(len(rows) + 1, dtype=np.int32)
        rpt[1:] = np.cumsum([len(r) for r in rows])
        col = np.concatenate(rows).astype(np.int32)
        val = rng.integers(-3, 4, col.size).astype(np.float64)
        return W.Csr(len(rows), ncols, rpt, col, val)
    return csr(a_rows, k), csr(b_rows, n)


@pytest.mark.parametrize("phase", [0, 1])
@pytest.mark.parametrize("kernel", range(len(ops.kernel_table(1)) - 1 if torch.cuda.is_available() else 0))
def test_multi_access_probe_each_hash_kernel(phase, kernel):
    # the read-then-swap probe (hash_access = 1, the access pattern the paper
    # compares its hashing against) gives the same C in every hash kernel
    A = W.rmat(11, 12, seed=71)
    cfg = forced(phase, kernel)
    cfg["hash_access"] = 1
    with ops.Handle(cfg) as h:
        check(A, A, gpu_product(A, A, h))
    B = W.random_csr(300, 200, 0.05, seed=72, duplicates=True, unsorted=True, integer_values=True)
    C = W.random_csr(200, 150, 0.08, seed=73, integer_values=True)
    with ops.Handle(cfg) as h:
        check(B, C, gpu_product(B, C, h), exact=True)


@pytest.mark.parametrize("kernel", range(len(ops.kernel_table(1)) if torch.cuda.is_available() else 0))
def test_contended_slot_updates_each_numeric_kernel(kernel):
    # every numeric kernel, many concurrent updates of one slot: the
    # compare-and-swap update must lose none of them (bit-exact sums)
    A, B = contended_product(60 + kernel)
    with ops.Handle(forced(1, kernel)) as h:
        got = gpu_product(A, B, h)
        bins = h.stats()["num_bins"]
    check(A, B, got, exact=True)
    assert bins[0] == A.rows


def narrow_rows(seed, m=160, width=700, per_row=(130, 240)):
    """A with rows of 130 to 240 entries inside a window of `width`
    columns that slides along the diagonal, integer values: C = A * I has
    the same narrow rows."""
    rng = np.random.default_rng(seed)
    n = m + width
    rows = []
    for i in range(m):
        k = rng.integers(per_row[0], per_row[1] + 1)
        rows.append(np.sort(rng.choice(width, k, replace=False) + i))
    rpt = np.zeros(m + 1, dtype=np.int32)
    rpt[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    A = W.Csr(m, n, rpt, col, rng.integers(-5, 6, col.size).astype(np.float64))
    I = W.Csr(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    return A, I


@pytest.mark.parametrize("kernel", range(len(ops.kernel_table(1)) if torch.cuda.is_available() else 0))
def test_narrow_rows_each_numeric_kernel(kernel):
    # rows whose columns span a few hundred: block-per-row kernels place
    # them by rank in a span bitmap, the others sort; C = A * I = A exactly
    A, I = narrow_rows(70 + kernel)
    cap = ops.kernel_table(1)[kernel][3]
    if cap != -1 and cap < 240:
        pytest.skip("rows larger than this kernel's tables")
    with ops.Handle(forced(1, kernel)) as h:
        got = gpu_product(A, I, h)
        bins = h.stats()["num_bins"]
    check(A, I, got, exact=True)
    assert bins[0] == A.rows


@pytest.mark.parametrize("extra", [0, 1])
def test_span_bitmap_boundary(extra):
    # the 512-slot kernel (64 threads) places a row of n entries by bitmap
    # rank when its span bitmap and prefix counts (2 words per 32 columns)
    # fit above the keys, n + 2 ceil(span / 32) <= 512, and sorts it
    # otherwise: rows of 182 entries spanning 5280 and 5281 columns
    table = ops.kernel_table(1)
    kernel = next(k for k, t in enumerate(table) if t[0] == 64 and t[2] == 512)
    rng = np.random.default_rng(80 + extra)
    last = 5279 + extra
    n = last + 65
    rows = []
    for i in range(24):
        mid = rng.choice(np.arange(1, last), 180, replace=False)
        rows.append(np.sort(np.concatenate([[0], mid, [last]])))
    rpt = np.zeros(len(rows) + 1, dtype=np.int32)
    rpt[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    A = W.Csr(len(rows), n, rpt, col, rng.integers(-5, 6, col.size).astype(np.float64))
    I = W.Csr(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    with ops.Handle(forced(1, kernel)) as h:
        got = gpu_product(A, I, h)
    check(A, I, got, exact=True)


@pytest.mark.parametrize("lanes", [1, 4, 32])
def test_fixed_lanes_per_b_row(lanes):
    A = W.rmat(10, 16, seed=8)
    cfg = ops.default_config()
    cfg["lanes_per_brow"] = lanes
    with ops.Handle(cfg) as h:
        check(A, A, gpu_product(A, A, h))


def test_bitmap_kernels_on_every_row():
    # every row through the bitmap kernels of both phases, including empty rows
    A = W.random_csr(500, 400, 0.02, seed=3, duplicates=True, unsorted=True)
    B = W.random_csr(400, 700, 0.03, seed=4)
    cfg = forced(0, len(ops.kernel_table(0)) - 1)
    cfg.update({k: v for k, v in forced(1, len(ops.kernel_table(1)) - 1).items()
                if k.startswith("num")})
    with ops.Handle(cfg) as h:
        check(A, B, gpu_product(A, B, h))


def test_wide_matrix_needs_several_bitmap_windows():
    # 4.5M columns: more than one shared-memory bitmap window in both phases
    rng = np.random.default_rng(9)
    K, N = 300, 4_500_000
    B = W._from_coo(K, N, np.repeat(np.arange(K), 40), rng.integers(0, N, size=K * 40),
                    rng.uniform(-1, 1, size=K * 40))
    A = W.random_csr(64, K, 0.3, seed=10)
    cfg = forced(0, len(ops.kernel_table(0)) - 1)
    cfg.update({k: v for k, v in forced(1, len(ops.kernel_table(1)) - 1).items()
                if k.startswith("num")})
    with ops.Handle(cfg) as h:
        check(A, B, gpu_product(A, B, h))
    with ops.Handle() as h:
        check(A, B, gpu_product(A, B, h))


def test_dense_row_goes_to_the_large_row_path(handle):
    # one row of A touches every row of B: n_prod far beyond any hash table
    K, N = 2000, 30000
    B = W.random_csr(K, N, 0.02, seed=12)
    r = np.concatenate([np.zeros(K, dtype=np.int64), [1, 2, 2]])
    c = np.concatenate([np.arange(K), [5, 7, 9]])
    A = W._from_coo(3, K, r, c, np.random.default_rng(1).uniform(-1, 1, size=r.size))
    got = gpu_product(A, B, handle)
    st = handle.stats()
    assert st["max_nprod"] > 30000
    check(A, B, got)


def _empty(rows, cols):
    return W.Csr(rows, cols, np.zeros(rows + 1, dtype=np.int32), np.zeros(0, dtype=np.int32),
                 np.zeros(0))


def test_empty_and_degenerate_shapes(handle):
    A = W.random_csr(50, 40, 0.1, seed=1)
    Z = _empty(40, 30)
    check(A, Z, gpu_product(A, Z, handle))                     # A * 0: all rows empty
    E = _empty(0, 40)
    B = W.random_csr(40, 5, 0.5, seed=2)
    check(E, B, gpu_product(E, B, handle))                     # no rows at all
    one = W.Csr(1, 1, np.array([0, 1], dtype=np.int32), np.array([0], dtype=np.int32),
                np.array([3.0]))
    check(one, one, gpu_product(one, one, handle), exact=True)


def test_row_windows(handle):
    A = W.rmat(12, 8, seed=21)
    dA = to_dev(A)
    for r0, r1 in ((0, 1), (100, 1733), (4000, 4096), (17, 17)):
        handle.symbolic(dA, dA, r0, r1)
        C = handle.numeric(dA, dA)
        handle.status()
        check(A, A, C.numpy(), r0=r0, r1=r1)


def test_preallocated_outputs(handle):
    A = W.rmat(10, 8, seed=22)
    dA = to_dev(A)
    nnz = handle.symbolic(dA, dA)
    col = torch.full((nnz + 5,), -7, dtype=torch.int32, device="cuda")
    val = torch.zeros(nnz + 5, dtype=torch.float64, device="cuda")
    C = handle.numeric(dA, dA, out=(col, val))
    handle.status()
    check(A, A, C.numpy())
    assert col[nnz:].tolist() == [-7] * 5


def test_galerkin_chain_with_int64_intermediate(handle):
    for s in (8, 9, 12):
        A, P, PT = W.galerkin_problem(s)
        AP = handle.multiply(to_dev(A), to_dev(P))      # AP.rpt is int64
        Ac = handle.multiply(to_dev(PT), AP)
        handle.status()
        rpt, col, val = Ac.numpy()
        if s % 2 == 0:
            L = W.laplacian_3d_7pt(s // 2)
            assert np.array_equal(rpt, L.rpt.astype(np.int64))
            assert np.array_equal(col, L.col)
            assert np.array_equal(val, 4.0 * L.val)
        else:
            APo = oracle.spgemm_csr(A, P)
            check(PT, W.Csr(APo.rows, APo.cols, APo.rpt, APo.col, APo.val), (rpt, col, val),
                  exact=True)


def test_errors_are_reported(handle):
    A = W.random_csr(10, 8, 0.3, seed=1)
    B = W.random_csr(9, 8, 0.3, seed=2)
    with pytest.raises(ops.SpgemmError) as e:
        handle.multiply(to_dev(A), to_dev(B))
    assert e.value.code == -2      # shape
    with pytest.raises(ops.SpgemmError) as e:
        handle.numeric(to_dev(A), to_dev(_empty(8, 8)))
    assert e.value.code in (-4, -2)   # no pending symbolic result
    bad = {"sym_kernel": [0, 0], "sym_range": [10, -1], "num_kernel": [0, 9],
           "num_range": [16, -1]}
    with pytest.raises(ops.SpgemmError):
        ops.Handle(bad)


def _sample_rows(C, rows):
    rpt = C.rpt.cpu().numpy()
    out = {}
    for i in rows:
        s, e = int(rpt[i]), int(rpt[i + 1])
        out[i] = (C.col[s:e].cpu().numpy(), C.val[s:e].cpu().numpy())
    return rpt, out


def _check_rows(A, B, sampled):
    for i, (col, val) in sampled.items():
        rpt, ocol, oval, ab = oracle.spgemm(A, B, i, i + 1)
        assert np.array_equal(col, ocol), i
        assert_values_close(val, oval, ab, what=f"row {i}")


def device_row_checks(C, r0, cnt_o, cs_o, vs_o, ab_o, what):
    """Every row of a device C (rows r0.. of the product) against the
    oracle's row checksums: size and sum of columns exactly, columns
    strictly increasing inside each row, and the sum of values within
    1e-12 of the row's sum of |a*b| plus the rounding of the two row sums
    (2 n u times the row's sum of |values|)."""
    rpt = C.rpt
    n = rpt.numel() - 1
    cnt = (rpt[1:] - rpt[:-1]).cpu().numpy()
    assert np.array_equal(cnt, cnt_o[r0:r0 + n]), f"{what}: row sizes"
    if C.nnz == 0:
        return
    col = C.col.long()
    csum = torch.zeros(C.nnz + 1, dtype=torch.int64, device=col.device)
    torch.cumsum(col, 0, out=csum[1:])
    cs = (csum[rpt[1:]] - csum[rpt[:-1]]).cpu().numpy()
    assert np.array_equal(cs, cs_o[r0:r0 + n]), f"{what}: column sums"
    inc = col[1:] > col[:-1]
    starts = torch.zeros(C.nnz, dtype=torch.bool, device=col.device)
    starts[rpt[1:-1][rpt[1:-1] < C.nnz]] = True
    assert bool((inc | starts[1:]).all()), f"{what}: columns not strictly increasing inside a row"
    del inc, starts, csum
    rowid = torch.repeat_interleave(torch.arange(n, device=col.device), rpt[1:] - rpt[:-1],
                                    output_size=C.nnz)
    vs = torch.zeros(n, dtype=torch.float64, device=col.device).index_add_(0, rowid, C.val).cpu().numpy()
    av = torch.zeros(n, dtype=torch.float64, device=col.device).index_add_(0, rowid, C.val.abs()).cpu().numpy()
    del rowid
    u = np.finfo(np.float64).eps / 2
    tol = 1e-12 * ab_o[r0:r0 + n] + 2 * cnt * u * av
    bad = np.abs(vs - vs_o[r0:r0 + n]) > tol
    assert not bad.any(), f"{what}: row value sums, first row {r0 + int(np.nonzero(bad)[0][0])}"


@pytest.mark.slow
def test_full_size_stencil27_128(handle):
    """The 27-point stencil on 128^3 (n = 2,097,152): closed-form totals and
    the whole C against the oracle element by element (254.8M entries)."""
    s = 128
    A = W.stencil27(s, seed=3)
    dA = to_dev(A)
    C = handle.multiply(dA, dA)
    handle.status()
    assert C.nnz == (5 * s - 6) ** 3 == 254840104
    assert handle.stats()["total_nprod"] == (9 * s - 10) ** 3 == 1489355288
    g_rpt, g_col, g_val = C.numpy()
    del C
    rpt, col, val, ab = oracle.spgemm(A, A, threads=oracle.max_threads())
    assert np.array_equal(g_rpt, rpt)
    assert np.array_equal(g_col, col)
    assert_values_close(g_val, val, ab)


@pytest.mark.slow
def test_full_size_rmat_2_20(handle):
    """R-MAT n = 2^20, degree 16, C ~ 9.7e9 entries (int64 C.rpt): every
    row's size, sum of columns and sum of values against the oracle's row
    checksums (C does not fit host memory, so rows are compared by these),
    computed in eight row slabs of about equal products so each slab's
    checks fit the device beside it, then the values of sampled and the
    heaviest rows in full."""
    from paper_2206_07244_gb300 import shard
    A = W.rmat(20, 16, seed=1)
    dA = to_dev(A)
    cnt_o, cs_o, vs_o, ab_o = oracle.row_checksums(A, A, threads=oracle.max_threads())
    assert int(cnt_o.sum()) > 2**31
    rng = np.random.default_rng(1)
    heavy = np.argsort(cnt_o)[-8:].tolist()
    rows = sorted(set(rng.integers(0, A.rows, 200).tolist()) | set(heavy))
    sampled = {}
    for r0, r1 in shard.slab_bounds(oracle.nprod(A, A), 8):
        handle.symbolic(dA, dA, r0, r1)
        C = handle.numeric(dA, dA)
        handle.status()
        device_row_checks(C, r0, cnt_o, cs_o, vs_o, ab_o, f"R-MAT 2^20 rows {r0}:{r1}")
        mine = [i for i in rows if r0 <= i < r1]
        _, got = _sample_rows(C, [i - r0 for i in mine])
        sampled.update({i + r0: v for i, v in got.items()})
        del C
        torch.cuda.empty_cache()
    assert len(sampled) == len(rows)
    _check_rows(A, A, sampled)
