"""Seeded synthetic CSR inputs for the row-wise SpGEMM C = A*B.

This module builds matrices only. It holds none of the multiplication's
arithmetic: it is the one module that both the CPU oracle tests and the CUDA
path's tests and benchmark draw their inputs from.

Every generator returns a ``Csr`` with int32 ``rpt`` (M+1), int32 ``col``
(nnz) and float64 ``val`` (nnz), rows sorted by column with no duplicates
(the CSR layout of Sec. 2.1.1) unless a generator is asked for duplicates or
unsorted columns on purpose. Random draws use numpy's PCG64 (``default_rng``),
which gives the same stream on every platform.

The paper measures on SuiteSparse matrices that are not available here; the
generators below stand in for them with the same kinds of structure: stencils
with a high compression ratio (Sec. 2.1.2), power-law graphs (R-MAT), banded
and block-diagonal matrices, and multigrid Galerkin operators.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Csr:
    rows: int
    cols: int
    rpt: np.ndarray  # int32 or int64, rows+1
    col: np.ndarray  # int32, nnz
    val: np.ndarray  # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def row(self, i: int):
        s, e = int(self.rpt[i]), int(self.rpt[i + 1])
        return self.col[s:e], self.val[s:e]

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.rows, self.cols), dtype=np.float64)
        for i in range(self.rows):
            c, v = self.row(i)
            for j, x in zip(c, v):
                d[i, j] += x
        return d


def _from_coo(rows: int, cols: int, r: np.ndarray, c: np.ndarray,
              v: np.ndarray, merge: bool = True) -> Csr:
    """Sort COO by (row, col); with ``merge`` duplicates are summed."""
    r = np.asarray(r, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    v = np.asarray(v, dtype=np.float64)
    key = r * np.int64(cols) + c
    order = np.argsort(key, kind="stable")
    key, v = key[order], v[order]
    if merge and key.size:
        uniq, first = np.unique(key, return_index=True)
        v = np.add.reduceat(v, first) if v.size else v
        key = uniq
    rr = key // np.int64(max(cols, 1))
    cc = key - rr * np.int64(max(cols, 1))
    counts = np.bincount(rr, minlength=rows).astype(np.int64)
    rpt = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(counts, out=rpt[1:])
    return Csr(rows, cols, rpt.astype(np.int32), cc.astype(np.int32),
               v.astype(np.float64))


def from_dense(d: np.ndarray) -> Csr:
    r, c = np.nonzero(d)
    return _from_coo(d.shape[0], d.shape[1], r, c, d[r, c])


def identity(n: int, scale: float = 1.0) -> Csr:
    idx = np.arange(n, dtype=np.int32)
    return Csr(n, n, np.arange(n + 1, dtype=np.int32), idx,
               np.full(n, scale, dtype=np.float64))


def permutation(perm: np.ndarray) -> Csr:
    """Row i holds a single 1.0 at column perm[i]."""
    perm = np.asarray(perm, dtype=np.int32)
    n = perm.size
    return Csr(n, n, np.arange(n + 1, dtype=np.int32), perm.copy(),
               np.ones(n, dtype=np.float64))


def tridiag_1d(n: int, diag: float = 2.0, off: float = -1.0) -> Csr:
    r, c, v = [], [], []
    i = np.arange(n)
    for d, x in ((-1, off), (0, diag), (1, off)):
        j = i + d
        m = (j >= 0) & (j < n)
        r.append(i[m]); c.append(j[m]); v.append(np.full(m.sum(), x))
    return _from_coo(n, n, np.concatenate(r), np.concatenate(c),
                     np.concatenate(v))


def laplacian_2d(nx: int, ny: int | None = None) -> Csr:
    """Dirichlet 5-point Laplacian on an nx*ny grid: 4 on the diagonal,
    -1 to each in-grid neighbour (point (x, y) is row y*nx + x)."""
    ny = nx if ny is None else ny
    n = nx * ny
    x = np.tile(np.arange(nx), ny)
    y = np.repeat(np.arange(ny), nx)
    i = np.arange(n)
    r, c, v = [i], [i], [np.full(n, 4.0)]
    for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        m = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
        r.append(i[m]); c.append(i[m] + dx + dy * nx); v.append(np.full(m.sum(), -1.0))
    return _from_coo(n, n, np.concatenate(r), np.concatenate(c),
                     np.concatenate(v))


def laplacian_3d_7pt(s: int) -> Csr:
    """Dirichlet 7-point Laplacian on an s^3 grid: 6 on the diagonal, -1 to
    each in-grid face neighbour (point (x, y, z) is row (z*s + y)*s + x)."""
    n = s ** 3
    i = np.arange(n, dtype=np.int64)
    x, y, z = i % s, (i // s) % s, i // (s * s)
    r, c, v = [i], [i], [np.full(n, 6.0)]
    for dx, dy, dz in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0),
                       (0, 0, -1), (0, 0, 1)):
        m = ((x + dx >= 0) & (x + dx < s) & (y + dy >= 0) & (y + dy < s)
             & (z + dz >= 0) & (z + dz < s))
        r.append(i[m]); c.append(i[m] + dx + dy * s + dz * s * s)
        v.append(np.full(int(m.sum()), -1.0))
    return _from_coo(n, n, np.concatenate(r), np.concatenate(c),
                     np.concatenate(v))


def stencil27(s: int, seed: int = 3) -> Csr:
    """27-point stencil on an s^3 grid: diagonal exactly 27.0, each in-grid
    off-diagonal neighbour uniform in [0.5, 1.5].

    Built row-major in column order directly (offsets sorted by dz, dy, dx),
    so no sort is needed even at s = 128 (55.7M entries)."""
    rng = np.random.default_rng(seed)
    n = s ** 3
    i = np.arange(n, dtype=np.int64)
    x, y, z = i % s, (i // s) % s, i // (s * s)
    counts = np.zeros(n, dtype=np.int64)
    masks = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                m = ((x + dx >= 0) & (x + dx < s) & (y + dy >= 0)
                     & (y + dy < s) & (z + dz >= 0) & (z + dz < s))
                masks.append((dx + dy * s + dz * s * s, dx == 0 and dy == 0 and dz == 0, m))
                counts += m
    rpt = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rpt[1:])
    nnz = int(rpt[-1])
    col = np.empty(nnz, dtype=np.int32)
    is_diag = np.zeros(nnz, dtype=bool)
    cursor = rpt[:-1].copy()
    for off, diag, m in masks:
        pos = cursor[m]
        col[pos] = (i[m] + off).astype(np.int32)
        if diag:
            is_diag[pos] = True
        cursor[m] += 1
    val = rng.uniform(0.5, 1.5, size=nnz)
    val[is_diag] = 27.0
    return Csr(n, n, rpt.astype(np.int32), col, val)


def rmat(scale: int, degree: int, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, values: str = "uniform") -> Csr:
    """Recursive-matrix (R-MAT) graph with n = 2^scale vertices.

    degree*n edges are drawn; each draw descends ``scale`` levels and picks
    the top-left quadrant with probability a, top-right (sets a column bit)
    with b, bottom-left (sets a row bit) with c and bottom-right with
    d = 1-a-b-c. Self-loops are kept, duplicates merged, and each surviving
    entry gets a value uniform in [-1, 1] from a second stream seeded
    (seed, 1). No noise and no vertex permutation."""
    n = 1 << scale
    m = degree * n
    rng = np.random.default_rng(seed)
    r = np.zeros(m, dtype=np.int64)
    cc = np.zeros(m, dtype=np.int64)
    t1, t2, t3 = a, a + b, a + b + c
    u = np.empty(m, dtype=np.float64)
    bit = np.empty(m, dtype=bool)
    tmp = np.empty(m, dtype=bool)
    for _ in range(scale):
        rng.random(out=u)
        np.left_shift(r, 1, out=r)
        np.left_shift(cc, 1, out=cc)
        np.greater_equal(u, t2, out=bit)          # bottom half: row bit
        r |= bit
        np.greater_equal(u, t1, out=tmp)          # top-right or bottom-right: column bit
        np.less(u, t2, out=bit)
        bit &= tmp
        np.greater_equal(u, t3, out=tmp)
        bit |= tmp
        cc |= bit
    del u, bit, tmp
    r <<= scale
    r |= cc
    del cc
    r.sort()
    keep = np.empty(r.size, dtype=bool)
    keep[:1] = True
    np.not_equal(r[1:], r[:-1], out=keep[1:])
    key = r[keep]
    del r, keep
    rr = key >> scale
    col = (key & (n - 1)).astype(np.int32)
    counts = np.bincount(rr, minlength=n)
    rpt = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rpt[1:])
    vrng = np.random.default_rng([seed, 1])
    if values == "uniform":
        val = vrng.uniform(-1.0, 1.0, size=key.size)
    else:
        val = np.ones(key.size)
    return Csr(n, n, rpt.astype(np.int32), col, val)


def banded(n: int, half_bw: int, seed: int) -> Csr:
    """Band matrix with |i-j| <= half_bw, values uniform in [-1, 1]."""
    rng = np.random.default_rng(seed)
    offs = np.arange(-half_bw, half_bw + 1)
    i = np.repeat(np.arange(n, dtype=np.int64), offs.size)
    j = i + np.tile(offs, n)
    m = (j >= 0) & (j < n)
    i, j = i[m], j[m]
    return _from_coo(n, n, i, j, rng.uniform(-1.0, 1.0, size=i.size), merge=False)


def block_diagonal(n: int, nblocks: int, mean_degree: float, seed: int) -> Csr:
    """Random block-diagonal matrix: n rows split into ``nblocks`` nearly
    equal diagonal blocks, each filled at a density that gives about
    ``mean_degree`` entries per row; values uniform in [-1, 1]."""
    rng = np.random.default_rng(seed)
    bounds = np.linspace(0, n, nblocks + 1).astype(np.int64)
    rs, cs = [], []
    for bi in range(nblocks):
        lo, hi = bounds[bi], bounds[bi + 1]
        w = hi - lo
        if w <= 0:
            continue
        k = int(round(mean_degree * w))
        rs.append(rng.integers(lo, hi, size=k))
        cs.append(rng.integers(lo, hi, size=k))
    r = np.concatenate(rs); c = np.concatenate(cs)
    out = _from_coo(n, n, r, c, np.zeros(r.size), merge=True)
    out.val = rng.uniform(-1.0, 1.0, size=out.nnz)
    return out


def random_csr(m: int, k: int, density: float, seed: int,
               duplicates: bool = False, unsorted: bool = False,
               integer_values: bool = False) -> Csr:
    """Uniform random sparse m*k matrix. With ``duplicates`` some entries
    appear twice in a row (the multiply must sum them); with ``unsorted`` the
    columns inside each row are shuffled. ``integer_values`` draws small
    integers so that every partial sum is exact in float64."""
    rng = np.random.default_rng(seed)
    cnt = rng.binomial(k, density, size=m) if k > 0 else np.zeros(m, dtype=np.int64)
    rows, cols = [], []
    for i in range(m):
        if cnt[i]:
            cs = rng.choice(k, size=cnt[i], replace=False)
            rows.append(np.full(cnt[i], i)); cols.append(cs)
    if rows:
        r = np.concatenate(rows); c = np.concatenate(cols)
    else:
        r = np.zeros(0, dtype=np.int64); c = np.zeros(0, dtype=np.int64)
    if integer_values:
        v = rng.integers(-4, 5, size=r.size).astype(np.float64)
    else:
        v = rng.uniform(-1.0, 1.0, size=r.size)
    out = _from_coo(m, k, r, c, v, merge=True)
    if duplicates and out.nnz:
        pick = rng.random(out.nnz) < 0.25
        rr = np.repeat(np.arange(m), np.diff(out.rpt.astype(np.int64)))
        r2 = np.concatenate([rr, rr[pick]])
        c2 = np.concatenate([out.col, out.col[pick]])
        if integer_values:
            v2 = np.concatenate([out.val, rng.integers(-4, 5, size=int(pick.sum())).astype(np.float64)])
        else:
            v2 = np.concatenate([out.val, rng.uniform(-1, 1, size=int(pick.sum()))])
        out = _from_coo(m, k, r2, c2, v2, merge=False)
    if unsorted and out.nnz:
        rpt = out.rpt.astype(np.int64)
        for i in range(m):
            s, e = rpt[i], rpt[i + 1]
            if e - s > 1:
                p = rng.permutation(e - s) + s
                out.col[s:e] = out.col[p]
                out.val[s:e] = out.val[p]
    return out


def aggregation_prolongator(s: int) -> Csr:
    """Piecewise-constant prolongator of 2x2x2 aggregation on an s^3 grid:
    fine point (x, y, z) maps to aggregate (x//2, y//2, z//2) of the
    ceil(s/2)^3 coarse grid, with value 1.0 (one entry per row)."""
    sc = (s + 1) // 2
    n = s ** 3
    i = np.arange(n, dtype=np.int64)
    x, y, z = i % s, (i // s) % s, i // (s * s)
    colv = ((z // 2) * sc + (y // 2)) * sc + (x // 2)
    return Csr(n, sc ** 3, np.arange(n + 1, dtype=np.int32),
               colv.astype(np.int32), np.ones(n, dtype=np.float64))


def transpose(a: Csr) -> Csr:
    """Explicit CSR transpose (a data-layout step of the generator)."""
    rr = np.repeat(np.arange(a.rows, dtype=np.int64), np.diff(a.rpt.astype(np.int64)))
    return _from_coo(a.cols, a.rows, a.col.astype(np.int64), rr, a.val, merge=False)


def galerkin_sides(count: int = 512, seed: int = 0, lo: int = 8, hi: int = 48) -> np.ndarray:
    """Grid sides of the batched multigrid workload: uniform integers in
    [lo, hi]."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=count)


def galerkin_problem(s: int):
    """(A, P, P^T) for one Galerkin product P^T (A P) on an s^3 grid."""
    A = laplacian_3d_7pt(s)
    P = aggregation_prolongator(s)
    return A, P, transpose(P)


def mlp_init(seed: int = 0) -> np.ndarray:
    """Initial parameters of the 6 -> 64 -> 64 -> 1 row-size predictor as one
    flat float64 vector (W1 6x64, b1, W2 64x64, b2, w3, b3): He-normal
    weights (std sqrt(2 / fan_in)), zero biases. These are the random numbers
    training starts from; both the CPU and the GPU side take them as input."""
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0.0, np.sqrt(2.0 / 6), size=(6, 64))
    w2 = rng.normal(0.0, np.sqrt(2.0 / 64), size=(64, 64))
    w3 = rng.normal(0.0, np.sqrt(2.0 / 64), size=64)
    return np.concatenate([w1.ravel(), np.zeros(64), w2.ravel(), np.zeros(64),
                           w3, np.zeros(1)])
