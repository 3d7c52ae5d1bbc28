"""Pins of the FP64 oracle of the learned preconditioner: finite-difference
gradients, the SPD property of M and the symmetry of its pattern."""
import numpy as np
import pytest

from oracle import gnn_fp64 as G
from paper_1607_01404_gb300 import workloads as wl


def _small():
    A = wl.weighted_grid(6, 2, seed=3)
    g = G.Graph(A.to_scipy())
    rng = np.random.default_rng(0)
    R = rng.standard_normal((g.n, 3))
    T = rng.standard_normal((g.n, 3))
    Y = rng.standard_normal((g.n, 2))
    X = rng.standard_normal((g.n, 2))
    return g, R, T, Y, X


def test_M_is_symmetric_spd_and_diagonally_dominant():
    A = wl.weighted_grid(10, 2, seed=5)
    g = G.Graph(A.to_scipy())
    p = G.init_params(1)
    m = G.forward(g, p)
    M = G.M_matrix(g, m).toarray()
    np.testing.assert_allclose(M, M.T, atol=0)
    off = M - np.diag(np.diag(M))
    assert np.all(np.abs(off).sum(axis=1) <= G.RHO * np.diag(M) * (1 + 1e-12))
    assert np.linalg.eigvalsh(M).min() > 0


def test_graph_matches_definition():
    A = wl.weighted_grid(5, 2, seed=2)
    S = A.to_scipy().toarray()
    g = G.Graph(A.to_scipy())
    C = S.T @ S
    np.testing.assert_allclose(g.C.toarray(), C, atol=1e-12)
    assert np.all(g.deg == (np.abs(C) > 0).sum(axis=1) - 1)
    E = g.E.toarray()
    d = np.diag(C)
    ref = C / np.sqrt(np.outer(d, d))
    np.fill_diagonal(ref, 0)
    np.testing.assert_allclose(E, ref, atol=1e-12)


@pytest.mark.parametrize("with_ritz", [False, True])
def test_gradient_matches_central_differences(with_ritz):
    g, R, T, Y, X = _small()
    p = G.init_params(7)
    theta = G.flatten(p)
    if with_ritz:
        loss, grads = G.loss_and_grad(g, p, R, T, Y, X)
    else:
        loss, grads = G.loss_and_grad(g, p, R, T)
    gflat = G.flatten(grads)
    rng = np.random.default_rng(1)
    idx = rng.choice(theta.size, size=40, replace=False)
    idx = np.concatenate([idx, [theta.size - 1, theta.size - 2, theta.size - 3]])  # the scalar parameters
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fp = G.loss_and_grad(g, G.unflatten(tp), R, T, *( (Y, X) if with_ritz else ()))[0]
        fm = G.loss_and_grad(g, G.unflatten(tm), R, T, *( (Y, X) if with_ritz else ()))[0]
        fd = (fp - fm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7, (i, fd, gflat[i])


def test_loss_is_scale_invariant():
    g, R, T, _, _ = _small()
    p = G.init_params(3)
    l1 = G.loss_and_grad(g, p, R, T)[0]
    l2 = G.loss_and_grad(g, p, R * 3.0, T * 0.5)[0]
    assert abs(l1 - l2) < 1e-12
    assert 0.0 <= l1 <= 1.0


def test_graph_keeps_cancelling_entries():
    # A^T A of [[1, 1], [1, -1]] is 2 I: the (0, 1) entry cancels but stays in the pattern
    import scipy.sparse as sp

    g = G.Graph(sp.csr_matrix(np.array([[1.0, 1.0], [1.0, -1.0]])))
    assert g.C.nnz == 4
    np.testing.assert_allclose(g.C.toarray(), 2 * np.eye(2), atol=0)
    assert g.deg.tolist() == [1.0, 1.0]
    assert np.all(g.e == 0)


def test_num_params_matches_library():
    from paper_1607_01404_gb300 import binding as B
    from paper_1607_01404_gb300 import build as BLD

    BLD.build()
    assert B.gnn_num_params() == G.n_params()
