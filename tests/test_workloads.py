"""The seeded generators build the matrices their definitions describe."""
import numpy as np
import pytest

from paper_1607_01404_gb300 import workloads as wl


def _D(N):
    D = np.zeros((N + 1, N))
    D[np.arange(N), np.arange(N)] = 1.0
    D[np.arange(1, N + 1), np.arange(N)] = -1.0
    return D


@pytest.mark.parametrize("N", [1, 2, 5, 8])
def test_grid2d_matches_kron(N):
    A = wl.grid_difference(N, 2)
    D, I = _D(N), np.eye(N)
    ref = np.vstack([np.kron(D, I), np.kron(I, D)])
    assert A.m == 2 * (N + 1) * N and A.n == N * N and A.nnz == 4 * N * N
    np.testing.assert_array_equal(A.to_scipy().toarray(), ref)


@pytest.mark.parametrize("N", [1, 3, 5])
def test_grid3d_matches_kron(N):
    A = wl.grid_difference(N, 3)
    D, I = _D(N), np.eye(N)
    ref = np.vstack([np.kron(np.kron(D, I), I), np.kron(np.kron(I, D), I), np.kron(np.kron(I, I), D)])
    assert A.nnz == 6 * N ** 3
    np.testing.assert_array_equal(A.to_scipy().toarray(), ref)


def test_config_sizes():
    # 2D N=32: nnz is 4 N^2 = 4096; 3D N=128: m = 3*129*128^2
    A = wl.grid_difference(32, 2)
    assert (A.m, A.n, A.nnz) == (2112, 1024, 4096)
    assert 3 * 129 * 128 ** 2 == 6340608


def test_csr_sorted_and_valid():
    for A in [wl.grid_difference(6, 3), wl.weighted_grid(7, 2, seed=3), wl.random_illconditioned(300, 100, 16, seed=2)]:
        rp, ci = A.rowptr.astype(np.int64), A.colidx
        assert rp[0] == 0 and rp[-1] == A.nnz and np.all(np.diff(rp) >= 0)
        assert ci.min() >= 0 and ci.max() < A.n
        for i in range(A.m):
            seg = ci[rp[i]:rp[i + 1]]
            assert np.all(np.diff(seg) > 0)


def test_weighted_grid_is_row_scaled():
    N = 6
    A0 = wl.grid_difference(N, 2).to_scipy().toarray()
    w = wl.lognormal_row_weights(A0.shape[0], seed=5)
    A = wl.grid_difference(N, 2, w).to_scipy().toarray()
    np.testing.assert_allclose(A, np.sqrt(w)[:, None] * A0, rtol=1e-15)
    assert w.min() >= 1e-3 and w.max() <= 1e3


def test_random_illconditioned_structure():
    A = wl.random_illconditioned(500, 120, 16, seed=4)
    S = A.to_scipy().tocsc()
    assert np.all(np.diff(S.indptr) == 16)  # 16 distinct rows per column
    B = wl.random_illconditioned(500, 120, 16, seed=4)
    np.testing.assert_array_equal(A.vals, B.vals)  # deterministic per seed
    C = wl.random_illconditioned(500, 120, 16, seed=5)
    assert not np.array_equal(A.vals, C.vals)
    # column scales lie in [1e-3, 1] times N(0,1) draws
    colmax = np.abs(S).max(axis=0).toarray().ravel()
    assert colmax.max() < 10.0
