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
    return g, rng.standard_normal((g.n, 5)), rng.standard_normal((g.n, 4))


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


def test_gradient_matches_central_differences():
    g, T0, X0 = _small()
    p = G.init_params(7)
    p["bs"] = np.array(0.8)
    theta = G.flatten(p)
    loss, grads = G.loss_and_grad(g, p, T0, X0, 3, 20)
    T, X = G.samples(g, G.forward(g, p), T0, X0, 3, 20)
    assert abs(G.loss_fixed_samples(g, p, T, X) - loss) < 1e-14
    gflat = G.flatten(grads)
    rng = np.random.default_rng(1)
    idx = rng.choice(theta.size, size=40, replace=False)
    idx = np.concatenate([idx, [theta.size - 1, theta.size - 2, theta.size - 3]])  # the scalar parameters
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (G.loss_fixed_samples(g, G.unflatten(tp), T, X) - G.loss_fixed_samples(g, G.unflatten(tm), T, X)) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7, (i, fd, gflat[i])


def test_dm_matches_central_differences():
    g, T, X = _small()
    m = G.forward(g, G.init_params(2))
    _, dm = G.loss_from_m(g, m, T, X)
    rng = np.random.default_rng(3)
    for k in rng.choice(m.size, size=25, replace=False):
        h = 1e-4 * abs(m[k]) + 1e-12
        mp, mm = m.copy(), m.copy()
        mp[k] += h
        mm[k] -= h
        fd = (G.loss_from_m(g, mp, T, X)[0] - G.loss_from_m(g, mm, T, X)[0]) / (2 * h)
        assert abs(fd - dm[k]) <= 1e-5 * abs(fd) + 1e-9 * np.abs(dm).max(), (k, fd, dm[k])


def _identity_m(g):
    return np.where(g.rows == g.indices, 1.0, 0.0)


def test_rayleigh_quotient_of_an_eigenvector():
    # x eigenvector of C with eigenvalue lam: rho(x) = lam x^T M x / x^T x
    g, _, _ = _small()
    lam, V = np.linalg.eigh(g.C.toarray())
    m = G.forward(g, G.init_params(4))
    M = G.M_matrix(g, m).toarray()
    X = V[:, [0, 3, 10]]
    rho, _ = G.rayleigh(g, m, X)
    np.testing.assert_allclose(rho, lam[[0, 3, 10]] * np.sum(X * (M @ X), axis=0), rtol=1e-10)


def test_loss_of_identity_on_eigenvectors_is_log_of_mean_eigenvalues():
    g, _, _ = _small()
    lam, V = np.linalg.eigh(g.C.toarray())
    hi, lo = [20, 25, 30, 35], [0, 1, 2]
    T, X = V[:, hi] * np.array([1.0, -2.0, 0.5, 3.0]), V[:, lo]
    L, _ = G.loss_from_m(g, _identity_m(g), T, X)
    assert abs(L - (np.log(lam[hi].mean()) - np.log(lam[lo].mean()))) < 1e-12


def test_samples_reach_the_extreme_eigenvalues_for_identity():
    # M = I: power steps converge to the top of the spectrum of C, smoothing
    # steps with omega = 1 / lam_max to the bottom
    g, T0, X0 = _small()
    lam = np.linalg.eigvalsh(g.C.toarray())
    m = _identity_m(g) / lam[-1]  # M C with spectrum in (0, 1]: no overflow over many power steps
    lam = lam / lam[-1]
    T, X = G.samples(g, m, T0[:, :1], X0[:, :1], 400, 4000)
    assert abs(G.rayleigh(g, m, T)[0][0] - lam[-1]) < 1e-6 * lam[-1]
    assert abs(G.rayleigh(g, m, X)[0][0] - lam[0]) < 1e-3 * lam[0]


def test_loss_is_scale_invariant():
    g, T0, X0 = _small()
    p = G.init_params(3)
    m = G.forward(g, p)
    T, X = G.samples(g, m, T0, X0, 3, 20)
    l1 = G.loss_from_m(g, m, T, X)[0]
    T2, X2 = G.samples(g, 2.5 * m, 3.0 * T0, 0.5 * X0, 3, 20)
    assert abs(G.loss_from_m(g, 2.5 * m, T2, X2)[0] - l1) < 1e-12
    assert l1 > 0


def test_edge_weights_follow_the_coupling_strength():
    g, _, _ = _small()
    p = G.init_params(0)
    for name in p:
        p[name] = np.zeros_like(p[name])
    p["bs"] = np.array(2.0)
    p["bd"] = np.array(1.0)
    m = G.forward(g, p)
    off = g.offdiag
    delta = np.log1p(np.e) / g.cdiag  # softplus(1) / c_ii
    mu = np.minimum(delta[g.rows], delta[g.indices])
    ref = 0.9 * np.tanh(2.0) * mu * np.abs(g.e) / np.maximum(g.wdeg[g.rows], g.wdeg[g.indices])
    np.testing.assert_allclose(m[off], ref[off], rtol=1e-13)
    np.testing.assert_allclose(m[~off], delta[g.rows[~off]], rtol=1e-13)


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
