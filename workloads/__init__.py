"""Seeded synthetic sparse-matrix generators.

This module is shared by the CPU oracle's tests, the GPU parity tests and the
benchmark.  It holds no arithmetic of the ordering method itself: it only makes
sparsity patterns (CSR, int32) with the shapes and degree structure of the
workloads the method is evaluated on.  Randomness comes from a counter-based
SplitMix64 stream implemented here with numpy uint64 arithmetic, so the same
seed gives the same matrix on every machine and numpy version.

The paper evaluates on SuiteSparse matrices (grid-like FEM meshes, web graphs,
circuit matrices); those are not available, so these generators stand in:

* ``grid_laplacian_2d`` / ``grid_laplacian_3d`` / ``stencil27``: regular
  stencil patterns (mesh-like matrices).
* ``powerlaw_symmetric``: Chung-Lu style random symmetric pattern whose expected
  row degrees follow a discrete power law (web-graph-like rows up to 2k).
* ``powerlaw_rectangular``: rectangular pattern with power-law column degrees
  (LP / term-document-like matrices).
* ``random_symmetric``: uniform random symmetric pattern with a given mean row
  count.
* ``batch_mix``: many independent matrices of uneven size, half grids and half
  random symmetric patterns.
* ``with_strengthened_diagonal``: an unsymmetric square pattern made from a
  symmetric one with a full diagonal (off-diagonal entries dropped at random,
  columns permuted at random), together with the perfect matching that the
  permuted diagonal forms (``meta["match"]``: row i's matched column).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea and Flood, 2014) on uint64 arrays."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def rand_u64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` pseudo-random 64-bit words of stream ``stream`` under ``seed``."""
    ctr = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = _mix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GOLDEN * np.uint64(stream + 1)],
                               dtype=np.uint64))[0]
        return _mix64(base + _GOLDEN * (ctr + np.uint64(1)))


def rand_uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (rand_u64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Matrix:
    """Sparsity pattern of an m x n matrix in CSR form (0-based, int32)."""

    name: str
    m: int
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def values(self) -> np.ndarray:
        """Laplacian-style values (diagonal 2*dim, off-diagonal -1). The ordering
        ignores values; they exist only so a user can assemble the matrix."""
        rows = np.repeat(np.arange(self.m, dtype=np.int64), np.diff(self.rowptr))
        diag = rows == self.colidx
        v = np.full(self.nnz, -1.0)
        v[diag] = float(self.meta.get("diag", 4.0))
        return v


def csr_from_coo(m: int, n: int, rows: np.ndarray, cols: np.ndarray, name: str,
                 meta: dict | None = None) -> Matrix:
    """CSR with sorted, de-duplicated column indices per row."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    key = np.sort(rows * n + cols)  # sort + adjacent dedup (the result np.unique gives, faster)
    if key.size:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    r = (key // n).astype(np.int64)
    c = (key % n).astype(np.int32)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=m), out=rowptr[1:])
    return Matrix(name, m, n, rowptr.astype(np.int32), c, meta or {})


def _stencil(dims: tuple[int, ...], offsets: list[tuple[int, ...]], name: str, diag: float) -> Matrix:
    """Regular stencil pattern on a grid with lexicographic (row-major) numbering.

    Built directly in sorted order: offsets are sorted by linear index delta, so
    the columns of every row come out ascending."""
    dims = tuple(int(s) for s in dims)
    N = int(np.prod(dims))
    strides = []
    acc = 1
    for s in reversed(dims):
        strides.append(acc)
        acc *= s
    strides = list(reversed(strides))
    offs = sorted(offsets, key=lambda o: sum(a * b for a, b in zip(o, strides)))
    coords = np.indices(dims, dtype=np.int32).reshape(len(dims), -1)
    cols = np.empty((N, len(offs)), dtype=np.int32)
    valid = np.ones((N, len(offs)), dtype=bool)
    lin = np.arange(N, dtype=np.int64)
    for j, o in enumerate(offs):
        ok = np.ones(N, dtype=bool)
        for a in range(len(dims)):
            c = coords[a] + o[a]
            ok &= (c >= 0) & (c < dims[a])
        valid[:, j] = ok
        cols[:, j] = (lin + sum(a * b for a, b in zip(o, strides))).astype(np.int32)
    counts = valid.sum(axis=1)
    rowptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = cols[valid]
    return Matrix(name, N, N, rowptr.astype(np.int32), colidx.astype(np.int32),
                  {"diag": diag, "grid": dims})


def grid_laplacian_2d(side: int) -> Matrix:
    """5-point Laplacian pattern on a side x side grid (values 4 / -1)."""
    offs = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]
    return _stencil((side, side), offs, f"grid2d_{side}x{side}", 4.0)


def grid_laplacian_3d(side: int) -> Matrix:
    """7-point Laplacian pattern on a side^3 grid (values 6 / -1)."""
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    return _stencil((side, side, side), offs, f"grid3d_{side}^3", 6.0)


def stencil27(side: int) -> Matrix:
    """27-point stencil pattern on a side^3 grid (side=100: 26,463,592 nonzeros)."""
    offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    return _stencil((side, side, side), offs, f"stencil27_{side}^3", 26.0)


def _powerlaw_degrees(count: int, exponent: float, dmin: int, dmax: int, seed: int, stream: int) -> np.ndarray:
    """Integer degrees drawn from P(d) ~ d^-exponent on [dmin, dmax]."""
    support = np.arange(dmin, dmax + 1, dtype=np.float64)
    pmf = support ** (-exponent)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    u = rand_uniform(seed, stream, count)
    idx = np.searchsorted(cdf, u, side="right")
    return (support[np.minimum(idx, len(support) - 1)]).astype(np.int64)


def powerlaw_symmetric(n: int, seed: int, exponent: float = 2.5, dmin: int = 4, dmax: int = 2000) -> Matrix:
    """Random structurally symmetric pattern with power-law expected degrees.

    Chung-Lu style: expected degrees w_i ~ d^-2.5 on [4, 2000] (mean ~10), about
    sum(w)/2 edges whose endpoints are drawn with probability proportional to w,
    self-loops dropped, duplicates merged, symmetrised, full diagonal added
    (about 11-12 nonzeros per row)."""
    w = _powerlaw_degrees(n, exponent, dmin, dmax, seed, 0).astype(np.float64)
    nedges = int(round(w.sum() / 2))
    cw = np.cumsum(w)
    cw /= cw[-1]
    a = np.searchsorted(cw, rand_uniform(seed, 1, nedges), side="right")
    b = np.searchsorted(cw, rand_uniform(seed, 2, nedges), side="right")
    a = np.minimum(a, n - 1)
    b = np.minimum(b, n - 1)
    keep = a != b
    a, b = a[keep], b[keep]
    diag = np.arange(n)
    rows = np.concatenate([a, b, diag])
    cols = np.concatenate([b, a, diag])
    return csr_from_coo(n, n, rows, cols, f"powerlaw_sym_{n}", {"diag": 1.0})


def powerlaw_rectangular(m: int, n: int, seed: int, exponent: float = 2.5, dmin: int = 6,
                         dmax: int = 2000) -> Matrix:
    """m x n pattern whose column degrees follow d^-2.5 on [6, 2000] (mean ~16);
    each column's rows are drawn uniformly (duplicates merged)."""
    deg = _powerlaw_degrees(n, exponent, dmin, dmax, seed, 0)
    cols = np.repeat(np.arange(n, dtype=np.int64), deg)
    rows = (rand_u64(seed, 1, cols.size) % np.uint64(m)).astype(np.int64)
    return csr_from_coo(m, n, rows, cols, f"powerlaw_rect_{m}x{n}", {"diag": 1.0})


def random_symmetric(n: int, nnz_per_row: float, seed: int, stream: int = 0) -> Matrix:
    """Uniform random symmetric pattern with about ``nnz_per_row`` entries per row
    (diagonal included)."""
    nedges = max(0, int(round(n * (nnz_per_row - 1.0) / 2.0)))
    r = rand_u64(seed, 2 * stream + 10, 2 * nedges)
    a = (r[:nedges] % np.uint64(n)).astype(np.int64)
    b = (r[nedges:] % np.uint64(n)).astype(np.int64)
    keep = a != b
    a, b = a[keep], b[keep]
    diag = np.arange(n)
    return csr_from_coo(n, n, np.concatenate([a, b, diag]), np.concatenate([b, a, diag]),
                        f"random_sym_{n}", {"diag": 1.0})


def random_pattern(m: int, n: int, nnz: int, seed: int, stream: int = 0) -> Matrix:
    """Uniform random (unsymmetric) m x n pattern with about ``nnz`` entries."""
    r = rand_u64(seed, 2 * stream + 20, 2 * nnz)
    rows = (r[:nnz] % np.uint64(max(m, 1))).astype(np.int64)
    cols = (r[nnz:] % np.uint64(max(n, 1))).astype(np.int64)
    return csr_from_coo(m, n, rows, cols, f"random_{m}x{n}")


def with_strengthened_diagonal(A: Matrix, keep: float, seed: int) -> Matrix:
    """Unsymmetric pattern with a known perfect matching: every off-diagonal
    entry of the square pattern A is kept with probability ``keep``, the
    diagonal is added, and the columns are permuted by a seeded random
    permutation pi (entry (i, j) -> (i, pi[j])).  meta["match"][i] = pi[i], the
    column that row i's diagonal entry moved to."""
    if A.m != A.n:
        raise ValueError("needs a square pattern")
    n = A.n
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(A.rowptr.astype(np.int64)))
    cols = A.colidx.astype(np.int64)
    u = rand_uniform(seed, 40, rows.size)
    off = rows != cols
    sel = off & (u < keep)
    rows, cols = np.concatenate([rows[sel], np.arange(n)]), np.concatenate([cols[sel], np.arange(n)])
    pi = np.argsort(rand_u64(seed, 41, n), kind="stable").astype(np.int64)
    B = csr_from_coo(n, n, rows, pi[cols], f"{A.name}_unsym", {"match": pi.astype(np.int32)})
    return B


def batch_mix(count: int, seed: int, nmin: int = 200, nmax: int = 20000) -> list[Matrix]:
    """``count`` independent matrices, n log-uniform in [nmin, nmax]; even-indexed
    ones are 2D 5-point grids (side round(sqrt(n))), odd-indexed ones uniform
    random symmetric patterns with mean row count uniform in [3, 30]."""
    u = rand_uniform(seed, 100, count)
    sizes = np.exp(np.log(nmin) + u * (np.log(nmax) - np.log(nmin)))
    rate = 3.0 + 27.0 * rand_uniform(seed, 101, count)
    mats = []
    for i in range(count):
        n = int(round(sizes[i]))
        if i % 2 == 0:
            side = max(2, int(round(np.sqrt(n))))
            mats.append(grid_laplacian_2d(side))
        else:
            mats.append(random_symmetric(n, float(rate[i]), seed, stream=1000 + i))
    return mats


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of an open-loop Poisson stream."""
    expected = int(rate_per_s * duration_s * 1.5 + 100)
    u = rand_uniform(seed, 200, expected)
    gaps = -np.log1p(-u) / rate_per_s
    t = np.cumsum(gaps)
    return t[t < duration_s]


# Workloads the method is measured on.  Each entry gives the matrix recipe, the
# hypergraph model, the layout dimension and the recursion limits.
CONFIGS = {
    "grid2d_64": dict(make=lambda: grid_laplacian_2d(64), model="symmetric", d=2,
                      min_part=64, max_depth=62, form="bbd"),
    "grid3d_64": dict(make=lambda: grid_laplacian_3d(64), model="symmetric", d=3,
                      min_part=64, max_depth=10, form="bbd"),
    "powerlaw_500k": dict(make=lambda: powerlaw_symmetric(500_000, seed=1), model="symmetric", d=3,
                          min_part=64, max_depth=10, form="bbd"),
    "rect_400k_300k": dict(make=lambda: powerlaw_rectangular(400_000, 300_000, seed=1), model="bipartite",
                           d=2, min_part=1, max_depth=6, form="sbd"),
}
