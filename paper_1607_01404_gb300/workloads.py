"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the SVD method: it only builds sparse
matrices in CSR form and seeded random blocks.  Every matrix family stands in
for a class of the paper's test problems (Sec. 4, Table 4), which are real
matrices that are not available here:

* grid-difference operators ``[D (x) I; I (x) D]`` in 2D and 3D, where ``D`` is
  the (N+1) x N forward-difference matrix (1 on the diagonal, -1 on the
  subdiagonal).  ``D^T D`` is the Dirichlet Laplacian ``tridiag(-1, 2, -1)``,
  so ``A^T A`` is the Laplacian of the paper's weak-scaling family (Sec. 4.3)
  and the singular values have a closed form;
* the same operators with log-normal per-row weights, ``A = W^{1/2} A0``;
* a tall random sparse matrix with 16 distinct nonzero rows per column and
  column scaling ``10^u``, u ~ U(-3, 0), standing in for the tall least-squares
  matrices of Table 4 (Rucci1, LargeRegFile, sls).

Random numbers that the method draws (the initial block of the first stage) are
produced here and passed to both implementations as inputs.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """A sparse matrix in compressed sparse row form (0-based, sorted columns)."""

    m: int
    n: int
    rowptr: np.ndarray  # int32, m + 1
    colidx: np.ndarray  # int32, nnz
    vals: np.ndarray  # float64, nnz
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.vals, self.colidx, self.rowptr), shape=(self.m, self.n))


def _from_coo(m: int, n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray, name: str) -> CSR:
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order]
    vals = vals[order]
    counts = np.bincount(rows, minlength=m)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 indices")
    return CSR(m, n, rowptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64), name)


def _difference_block(N: int, dims: int, axis: int):
    """COO of the block of A that differences along ``axis`` of an N^dims grid.

    Rows enumerate an N^dims grid extended to N+1 points along ``axis``; the
    row (.., i, ..) holds +1 at grid column (.., i, ..) when i < N and -1 at
    (.., i-1, ..) when i >= 1.
    """
    shape_r = [N] * dims
    shape_r[axis] = N + 1
    nrows = int(np.prod(shape_r))
    idx = np.indices(shape_r).reshape(dims, -1)  # row multi-indices, C order
    rows_all = np.arange(nrows, dtype=np.int64)
    strides = [N ** (dims - 1 - d) for d in range(dims)]
    i_ax = idx[axis]
    base = np.zeros(nrows, dtype=np.int64)
    for d in range(dims):
        if d != axis:
            base += idx[d].astype(np.int64) * strides[d]
    plus = i_ax < N
    minus = i_ax >= 1
    r = np.concatenate([rows_all[plus], rows_all[minus]])
    c = np.concatenate([base[plus] + i_ax[plus].astype(np.int64) * strides[axis],
                        base[minus] + (i_ax[minus].astype(np.int64) - 1) * strides[axis]])
    v = np.concatenate([np.ones(int(plus.sum())), -np.ones(int(minus.sum()))])
    return nrows, r, c, v


def grid_difference(N: int, dims: int, row_weights: np.ndarray | None = None, name: str = "") -> CSR:
    """``A = W^{1/2} [D(x)I(x)I; I(x)D(x)I; I(x)I(x)D]`` (dims = 2 or 3) on an N^dims grid.

    m = dims (N+1) N^(dims-1) rows, n = N^dims columns, nnz = 2 dims N^dims.
    """
    rows, cols, vals = [], [], []
    off = 0
    for axis in range(dims):
        nr, r, c, v = _difference_block(N, dims, axis)
        rows.append(r + off)
        cols.append(c)
        vals.append(v)
        off += nr
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    m, n = off, N ** dims
    if row_weights is not None:
        row_weights = np.asarray(row_weights, dtype=np.float64)
        assert row_weights.shape == (m,)
        v = v * np.sqrt(row_weights[r])
    return _from_coo(m, n, r, c, v, name or f"grid{dims}d_N{N}")


def lognormal_row_weights(m: int, seed: int, sigma: float = 1.5, lo: float = 1e-3, hi: float = 1e3) -> np.ndarray:
    """Per-row (per grid edge) weights ``clip(exp(sigma z), lo, hi)``, z ~ N(0, 1)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5EED, seed]))
    return np.clip(np.exp(sigma * rng.standard_normal(m)), lo, hi)


def weighted_grid(N: int, dims: int, seed: int) -> CSR:
    m = dims * (N + 1) * N ** (dims - 1)
    return grid_difference(N, dims, lognormal_row_weights(m, seed), name=f"wgrid{dims}d_N{N}_s{seed}")


def random_illconditioned(m: int, n: int, per_col: int = 16, seed: int = 0, umin: float = -3.0, umax: float = 0.0) -> CSR:
    """Tall random sparse matrix: ``per_col`` distinct uniform rows per column,
    N(0,1) values, column j scaled by ``10^u_j`` with u_j ~ U(umin, umax)."""
    if per_col > m:
        raise ValueError("per_col > m")
    rng = np.random.default_rng(np.random.SeedSequence([0xC0FFEE, seed]))
    rows = rng.integers(0, m, size=(n, per_col), dtype=np.int64)
    while True:  # redraw duplicates inside a column until all rows are distinct
        rows.sort(axis=1)
        dup = np.zeros_like(rows, dtype=bool)
        dup[:, 1:] = rows[:, 1:] == rows[:, :-1]
        nd = int(dup.sum())
        if nd == 0:
            break
        rows[dup] = rng.integers(0, m, size=nd, dtype=np.int64)
    vals = rng.standard_normal((n, per_col))
    u = rng.uniform(umin, umax, size=n)
    vals *= (10.0 ** u)[:, None]
    cols = np.repeat(np.arange(n, dtype=np.int64), per_col)
    return _from_coo(m, n, rows.reshape(-1), cols, vals.reshape(-1), f"randill_{m}x{n}_s{seed}")


def start_block(n: int, b: int, seed: int = 0) -> np.ndarray:
    """Seeded N(0,1) initial block for the first stage, n x b, column-major (Fortran order)."""
    rng = np.random.default_rng(np.random.SeedSequence([0xB10C, seed]))
    return np.asfortranarray(rng.standard_normal((n, b)))


def dense_block(rows: int, cols: int, seed: int = 0) -> np.ndarray:
    """Seeded N(0,1) dense block, row-major, for per-kernel parity tests."""
    rng = np.random.default_rng(np.random.SeedSequence([0xD0E5, seed]))
    return rng.standard_normal((rows, cols))


# Named workloads (sizes of the paper-shaped synthetic problems).
def workload(name: str) -> tuple[CSR, dict]:
    """Return (A, task) for a named workload; task holds k, target and block size."""
    if name == "grid2d_N32":  # 2112 x 1024, closed-form spectrum
        return grid_difference(32, 2), dict(k=5, b=1)
    if name == "grid3d_N128":  # 6,340,608 x 2,097,152, closed-form spectrum
        return grid_difference(128, 3), dict(k=10, b=4, target="smallest")
    if name == "randill_1e6x5e5":
        return random_illconditioned(1_000_000, 500_000, 16, seed=0), dict(k=10, b=4)
    if name == "wgrid2d_N256":
        return weighted_grid(256, 2, seed=10000), dict(k=10, b=4, target="smallest")
    if name == "wgrid3d_N96":
        return weighted_grid(96, 3, seed=10000), dict(k=20, b=8, target="smallest")
    raise KeyError(name)
