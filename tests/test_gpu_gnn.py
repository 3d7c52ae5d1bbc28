"""GPU parity of the learned preconditioner: graph of C = A^T A, forward M
values and loss gradients against the FP64 oracle (oracle/gnn_fp64.py)."""
import numpy as np
import pytest

from oracle import gnn_fp64 as G
from paper_1607_01404_gb300 import binding as B
from paper_1607_01404_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# FP32 network: forward values within 2e-4 of the row's diagonal, gradients
# within 2e-3 of the gradient norm (FP32 products of depth ~10 layers).
M_TOL = 2e-4
G_TOL = 2e-3


def _cases():
    return [
        ("wgrid2d_20", wl.weighted_grid(20, 2, seed=7)),
        ("grid3d_9", wl.grid_difference(9, 3)),
        ("randill_300x170", wl.random_illconditioned(300, 170, per_col=4, seed=2)),
    ]


def _gnn(A):
    return B.Gnn(A.rowptr, A.colidx, A.vals, A.m, A.n)


def _theta(seed):
    p = G.init_params(seed)
    rng = np.random.default_rng(100 + seed)
    # non-zero biases so that every head term is exercised
    p["we"] = np.array(0.3)
    p["bs"] = np.array(-0.2)
    for l in range(G.LAYERS):
        p[f"b_{l}"] = 0.1 * rng.standard_normal(G.WIDTH)
    th = G.flatten(p).astype(np.float32)
    return th, G.unflatten(th.astype(np.float64))


@pytest.mark.parametrize("name,A", _cases())
def test_graph_pattern_bit_exact(name, A):
    g = _gnn(A)
    ref = G.Graph(A.to_scipy())
    rp, ci = g.pattern()
    assert g.n == ref.n and g.nnz == ref.C.nnz
    np.testing.assert_array_equal(rp, ref.indptr)
    np.testing.assert_array_equal(ci, ref.indices)
    g.close()


def test_graph_of_wide_matrix():
    A = wl.random_illconditioned(120, 200, per_col=3, seed=5)
    g = _gnn(A)
    ref = G.Graph(A.to_scipy())
    rp, ci = g.pattern()
    assert g.n == 200
    np.testing.assert_array_equal(rp, ref.indptr)
    np.testing.assert_array_equal(ci, ref.indices)
    th, p = _theta(1)
    m = g.forward(th)
    mr = G.forward(ref, p)
    diag = np.repeat(mr[ref.rows == ref.indices], np.diff(ref.indptr))
    assert np.max(np.abs(m - mr) / diag) < M_TOL


@pytest.mark.parametrize("name,A", _cases())
def test_forward_matches_oracle_and_is_spd(name, A):
    g = _gnn(A)
    ref = G.Graph(A.to_scipy())
    for seed in (0, 3):
        th, p = _theta(seed)
        m = g.forward(th).astype(np.float64)
        mr = G.forward(ref, p)
        diag = np.repeat(mr[ref.rows == ref.indices], np.diff(ref.indptr))
        err = np.abs(m - mr) / diag
        assert err.max() < M_TOL, (name, seed, err.max())
        # the GPU's own M is symmetric and strictly diagonally dominant
        M = G.M_matrix(ref, m)
        assert abs(M - M.T).max() == 0
        d = M.diagonal()
        off = np.asarray(abs(M).sum(axis=1)).ravel() - d
        assert np.all(d > 0) and np.all(off < d)
    g.close()


@pytest.mark.parametrize("name,A", _cases())
def test_loss_and_gradient_match_oracle(name, A):
    g = _gnn(A)
    ref = G.Graph(A.to_scipy())
    rng = np.random.default_rng(11)
    n = ref.n
    R, T = rng.standard_normal((n, 5)), rng.standard_normal((n, 5))
    Y, X = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    th, p = _theta(2)
    for with_q in (False, True):
        args = (R, T, Y, X) if with_q else (R, T)
        L, grad = g.loss_grad(th, *args)
        Lr, gr = G.loss_and_grad(ref, p, *args)
        gr = G.flatten(gr)
        assert abs(L - Lr) < 1e-5 * max(1.0, abs(Lr)), (L, Lr)
        err = np.linalg.norm(grad - gr) / np.linalg.norm(gr)
        assert err < G_TOL, (name, with_q, err)
    g.close()


def test_gradient_is_a_descent_direction_and_adam_steps():
    A = wl.weighted_grid(16, 2, seed=1)
    g = _gnn(A)
    rng = np.random.default_rng(5)
    R, T = rng.standard_normal((g.n, 4)), rng.standard_normal((g.n, 4))
    th, _ = _theta(4)
    L0, grad = g.loss_grad(th, R, T)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    th1 = th.copy()
    g.adam(th1, grad, m, v, 1, 1e-3)
    # first Adam step: m = 0.1 g, v = 0.001 g^2, update = lr * sign-like ratio
    mh = (0.1 * grad) / 0.1
    vh = (0.001 * grad * grad) / 0.001
    ref = th.astype(np.float64) - 1e-3 * mh / (np.sqrt(vh) + 1e-8)
    np.testing.assert_allclose(th1, ref, rtol=1e-5, atol=1e-7)
    L1, _ = g.loss_grad(th1, R, T)
    assert L1 < L0
    g.close()


def test_rejects_bad_arguments():
    A = wl.weighted_grid(6, 2, seed=1)
    g = _gnn(A)
    th, _ = _theta(0)
    R = np.zeros((g.n, 9))
    with pytest.raises(B.SvdsError):
        g.loss_grad(th, R, R)  # at most 8 pairs per call
    with pytest.raises(ValueError):
        g.forward(th[:-1])
    g.close()
