"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module only *builds inputs*: sparse matrices in CRS form (int32 row
pointer, int32 column index, float64 value) and dense vectors drawn from a
counter-based generator.  It holds none of the matrix-power arithmetic, no
BFS, no permutation and no grouping, so that the oracle (``oracle/``) and the
GPU library can both consume the same inputs without sharing method code.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw ``i`` of stream ``seed`` is ``mix(seed + (i+1)*GOLDEN)``.
A uniform double in [0,1) is ``(z >> 11) * 2**-53``.

Matrix families follow the workloads of the paper: the 2d-7pt worked example
of Sec. 4.1 (Fig. 3), 2D/3D Laplacian stencils (Tab. 3 "order-2" heat
matrix), higher-order star stencils (Tab. 3 order-4/6), the HPCG 27-point
stencil (Tab. 2) and the 3D Anderson Hamiltonian of Sec. 7.
Lexicographic numbering with x fastest is used throughout.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class CSR:
    """A square sparse matrix in CRS layout (host numpy arrays)."""

    def __init__(self, n, rowptr, col, val, name=""):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.name = name
        assert self.rowptr.shape == (self.n + 1,)
        assert self.col.shape == self.val.shape == (int(self.rowptr[-1]),)

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def __repr__(self):
        return f"CSR({self.name!r}, n={self.n}, nnz={self.nnz})"


# ---------------------------------------------------------------- random numbers
def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset..offset+count-1 of SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, count)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on two streams of uniforms."""
    u1 = uniform01(seed, count, 0)
    u2 = uniform01(seed, count, count)
    u1 = np.where(u1 <= 0.0, 2.0 ** -53, u1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def random_vector(n: int, seed: int = 1234, nrhs: int = 1) -> np.ndarray:
    """x ~ U[-1, 1]; shape (n,) or row-major (n, nrhs)."""
    v = uniform(seed, n * nrhs)
    return v if nrhs == 1 else v.reshape(n, nrhs)


def integer_vector(n: int, seed: int = 99) -> np.ndarray:
    """x with entries in {-1, 0, 1} (for the exact integer-valued checks)."""
    z = splitmix64(seed, n)
    return ((z % np.uint64(3)).astype(np.int64) - 1).astype(np.float64)


# ---------------------------------------------------------------- stencil builder
def _grid_stencil(dims, offsets, values, periodic=False, name=""):
    """CRS of a stencil on a grid of shape `dims` (x fastest).

    offsets: list of integer tuples (dx, dy[, dz]); values: matching list of
    floats or callables(row_ids) -> per-row values.  Rows are grid points;
    columns within each row are sorted ascending.
    """
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    n = int(np.prod(dims))
    ids = np.arange(n, dtype=np.int64)
    coords = []
    rem = ids
    for d in dims:
        coords.append(rem % d)
        rem = rem // d
    strides = [int(np.prod(dims[:k])) for k in range(nd)]
    cols = np.empty((n, len(offsets)), dtype=np.int64)
    vals = np.empty((n, len(offsets)), dtype=np.float64)
    ok = np.ones((n, len(offsets)), dtype=bool)
    for j, (off, v) in enumerate(zip(offsets, values)):
        c = np.zeros(n, dtype=np.int64)
        valid = np.ones(n, dtype=bool)
        for k in range(nd):
            q = coords[k] + off[k]
            if periodic:
                q = q % dims[k]
            else:
                valid &= (q >= 0) & (q < dims[k])
            c += q * strides[k]
        cols[:, j] = np.where(valid, c, -1)
        vals[:, j] = v(ids) if callable(v) else v
        ok[:, j] = valid
    # sort each row's entries by column (padding -1 entries go first, then dropped)
    order = np.argsort(np.where(ok, cols, -1), axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    vals = np.take_along_axis(vals, order, axis=1)
    ok = np.take_along_axis(ok, order, axis=1)
    counts = ok.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if periodic:
        # duplicates appear when a dimension is < 3 with wrap-around; merge them
        assert all(d >= 3 for d in dims), "periodic stencils need every dim >= 3"
    return CSR(n, rowptr, cols[ok], vals[ok], name)


def laplace1d(n: int) -> CSR:
    """1D Dirichlet Laplacian: diagonal 2, off-diagonals -1."""
    return _grid_stencil((n,), [(-1,), (0,), (1,)], [-1.0, 2.0, -1.0], name=f"laplace1d-{n}")


def laplace2d(nx: int, ny: int | None = None) -> CSR:
    """2D 5-point Dirichlet Laplacian: diagonal 4, off-diagonals -1."""
    ny = nx if ny is None else ny
    offs = [(0, -1), (-1, 0), (0, 0), (1, 0), (0, 1)]
    vals = [-1.0, -1.0, 4.0, -1.0, -1.0]
    return _grid_stencil((nx, ny), offs, vals, name=f"laplace2d-{nx}x{ny}")


def laplace3d(n: int) -> CSR:
    """3D 7-point Dirichlet Laplacian: diagonal 6, off-diagonals -1 (Tab. 3 order-2)."""
    offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    vals = [-1.0] * 3 + [6.0] + [-1.0] * 3
    return _grid_stencil((n, n, n), offs, vals, name=f"laplace3d-{n}")


def stencil2d_7pt(nx: int, ny: int | None = None) -> CSR:
    """The 2d-7pt stencil of the paper's worked example (Sec. 4.1, Fig. 3).

    Neighbours (x+-1, y), (x, y+-1), (x+1, y-1), (x-1, y+1) plus the centre.
    Values: centre 6, neighbours -1 (only the pattern matters for levels).
    """
    ny = nx if ny is None else ny
    offs = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1), (1, -1), (-1, 1)]
    vals = [6.0] + [-1.0] * 6
    return _grid_stencil((nx, ny), offs, vals, name=f"2d7pt-{nx}x{ny}")


_FD2 = {  # central second-derivative weights of spatial order 2, 4, 6
    1: [1.0, -2.0],
    2: [-1.0 / 12, 4.0 / 3, -5.0 / 2],
    3: [1.0 / 90, -3.0 / 20, 3.0 / 2, -49.0 / 18],
}


def star3d(n: int, radius: int) -> CSR:
    """Negative 3D Laplacian from central differences of order 2*radius
    (Tab. 3 order-2/4/6 heat matrices on an n^3 grid, Dirichlet)."""
    w = _FD2[radius]  # w[0] is the outermost weight, w[-1] the centre
    offs, vals = [], []
    for ax in range(3):
        for s in range(-radius, radius + 1):
            if s == 0:
                continue
            o = [0, 0, 0]
            o[ax] = s
            offs.append(tuple(o))
            vals.append(-w[radius - abs(s)])
    offs.append((0, 0, 0))
    vals.append(-3.0 * w[-1])
    return _grid_stencil((n, n, n), offs, vals, name=f"star3d-r{radius}-{n}")


def box27(n: int) -> CSR:
    """27-point stencil (HPCG matrix): diagonal 26, off-diagonals -1."""
    offs, vals = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                offs.append((dx, dy, dz))
                vals.append(26.0 if (dx, dy, dz) == (0, 0, 0) else -1.0)
    return _grid_stencil((n, n, n), offs, vals, name=f"box27-{n}")


def anderson3d(n: int, W: float = 16.5, seed: int = 42, periodic: bool = True) -> CSR:
    """3D Anderson Hamiltonian (Sec. 7): hopping -1 to the 6 nearest
    neighbours, on-site disorder uniform in [-W/2, W/2] from `seed`."""
    N = n ** 3
    eps = uniform(seed, N, -W / 2.0, W / 2.0)
    offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    vals = [-1.0] * 3 + [lambda ids: eps[ids]] + [-1.0] * 3
    return _grid_stencil((n, n, n), offs, vals, periodic=periodic,
                         name=f"anderson3d-{n}{'-pbc' if periodic else ''}")


def diagonal(d: np.ndarray) -> CSR:
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    return CSR(n, np.arange(n + 1), np.arange(n), d, name=f"diag-{n}")


def from_dense(A: np.ndarray, name="dense") -> CSR:
    """CRS of the nonzero pattern of a dense matrix (stored entries = nonzeros)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    np.cumsum(rowptr, out=rowptr)
    return CSR(n, rowptr, cols, A[rows, cols], name=name)


def random_sparse(n: int, density: float, seed: int, symmetric: bool = True,
                  diag: bool = True) -> CSR:
    """Random sparse matrix (dense-built; for small n only)."""
    u = uniform01(seed, n * n).reshape(n, n)
    v = uniform(seed + 1, n * n).reshape(n, n)
    mask = u < density
    if symmetric:
        mask = np.triu(mask, 1)
        mask = mask | mask.T
        v = np.triu(v, 1)
        v = v + v.T
    if diag:
        np.fill_diagonal(mask, True)
        np.fill_diagonal(v, 1.0 + uniform01(seed + 2, n))
    A = np.where(mask, v, 0.0)
    if diag:
        np.fill_diagonal(A, np.diag(v))
    return from_dense(A, name=f"rand{'sym' if symmetric else ''}-{n}-{density}-{seed}")


# ---------------------------------------------------------------- irregular graphs
def zipf_degrees(n: int, seed: int, s: float = 2.0, base: int = 8, cap: int = 500) -> np.ndarray:
    """Target degrees min(cap, base + Z), Z ~ Zipf(s) on 1..cap-base (finite
    support, inverse-CDF sampling); mean about 12 for s = 2, base = 8."""
    k = np.arange(1, cap - base + 1, dtype=np.float64)
    cdf = np.cumsum(k ** -s)
    cdf /= cdf[-1]
    z = np.searchsorted(cdf, uniform01(seed, n), side="right") + 1
    return np.minimum(cap, base + z).astype(np.int64)


def _symmetric_from_pairs(n: int, u: np.ndarray, v: np.ndarray, wseed: int, name: str) -> CSR:
    """Symmetric CRS from distinct upper-triangle pairs u < v sorted by (u, v):
    a_uv = a_vu ~ N(0,1) from stream wseed, a_ii = sum_j |a_ij| + 1.  Rows come
    out with ascending columns."""
    w = normal(wseed, u.size)
    absw = np.abs(w)
    lower_order = np.argsort(v * n + u)             # lower triangle entries (row v, col u) in row order
    lu, lv, lw = v[lower_order], u[lower_order], w[lower_order]
    cnt_up = np.bincount(u, minlength=n)
    cnt_lo = np.bincount(lu, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_lo + 1 + cnt_up, out=rowptr[1:])
    nnz = int(rowptr[-1])
    col = np.empty(nnz, dtype=np.int64)
    val = np.empty(nnz, dtype=np.float64)
    first_lo = np.concatenate([[0], np.cumsum(cnt_lo)[:-1]])
    pos_lo = rowptr[:-1][lu] + (np.arange(lu.size) - first_lo[lu])
    col[pos_lo], val[pos_lo] = lv, lw
    pos_d = rowptr[:-1] + cnt_lo
    col[pos_d] = np.arange(n)
    val[pos_d] = np.bincount(u, absw, minlength=n) + np.bincount(v, absw, minlength=n) + 1.0
    first_up = np.concatenate([[0], np.cumsum(cnt_up)[:-1]])
    pos_up = pos_d[u] + 1 + (np.arange(u.size) - first_up[u])
    col[pos_up], val[pos_up] = v, w
    return CSR(n, rowptr, col, val, name=name)


def zipf_graph(n: int, seed: int) -> CSR:
    """Random symmetric sparse matrix with Zipf-distributed row degrees
    (configuration model): half-edges are paired at random, self-loops and
    duplicate pairs dropped; a_ij = a_ji ~ N(0,1) and a_ii = sum_j |a_ij| + 1
    (diagonally dominant).  Rows come out with ascending columns.
    Deterministic in (n, seed) (PCG64 of numpy for the pairing)."""
    deg = zipf_degrees(n, seed)
    half = np.repeat(np.arange(n, dtype=np.int64), deg)
    if half.size % 2:
        half = half[:-1]
    half = np.random.default_rng(seed).permutation(half)
    u, v = half[0::2], half[1::2]
    keep = u != v
    u, v = np.minimum(u[keep], v[keep]), np.maximum(u[keep], v[keep])
    key = np.sort(u * n + v)                        # upper triangle, sorted by (row u, col v)
    key = key[np.concatenate([[True], key[1:] != key[:-1]])]   # drop duplicate pairs
    return _symmetric_from_pairs(n, key // n, key % n, seed + 2, f"zipf-{n}-{seed}")


def random_geometric_graph(n: int, dim: int, degree: float, seed: int) -> CSR:
    """Random geometric graph as a symmetric matrix: n points uniform in the
    unit cube [0,1)^dim (coordinates from SplitMix64 stream seed), an edge
    between every pair closer than r, with r set so that an interior point has
    `degree` neighbours on average (n * V_dim * r^dim = degree).  The points
    are numbered in draw order, so the natural numbering has no locality;
    values as in zipf_graph (stream seed + 1)."""
    from scipy.spatial import cKDTree
    vol = {2: np.pi, 3: 4.0 * np.pi / 3.0}[dim]
    r = (degree / (n * vol)) ** (1.0 / dim)
    pts = uniform01(seed, n * dim).reshape(n, dim)
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray").astype(np.int64)
    u, v = np.minimum(pairs[:, 0], pairs[:, 1]), np.maximum(pairs[:, 0], pairs[:, 1])
    key = np.sort(u * n + v)
    return _symmetric_from_pairs(n, key // n, key % n, seed + 1, f"rgg{dim}d-{n}-{seed}")


def batch_workload(count: int = 64, seed0: int = 1000, n_lo: int = 20_000, n_hi: int = 2_000_000):
    """The batched workload: `count` Zipf graphs, matrix m with seed seed0+m,
    N ~ U[n_lo, n_hi], nrhs ~ U{1..16}, p ~ U{2..10}.  Returns a list of
    (CSR, nrhs, p)."""
    out = []
    for m in range(count):
        z = splitmix64(seed0 + m, 3)
        n = n_lo + int(z[0] % np.uint64(n_hi - n_lo + 1))
        nrhs = 1 + int(z[1] % np.uint64(16))
        p = 2 + int(z[2] % np.uint64(9))
        out.append((zipf_graph(n, seed0 + m), nrhs, p))
    return out
