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


# ---------------------------------------------------------------------------
# Pin of the message-passing layers and heads: the network recomputed node by
# node with plain Python loops from the definition (graph of A^T A, features,
# h' = relu(h W1 + (E h) W2 + b) for 4 layers, node and edge heads, M), with
# non-zero parameters so that every term reaches the output.
# ---------------------------------------------------------------------------
def _forward_by_loops(Ad, params):
    """Ad: small dense A (list of rows).  Returns (list of h^l, {(i, j): m_ij})."""
    import math

    mrows, n = len(Ad), len(Ad[0])
    C = [[sum(Ad[r][i] * Ad[r][j] for r in range(mrows)) for j in range(n)] for i in range(n)]
    pat = [[any(Ad[r][i] != 0 and Ad[r][j] != 0 for r in range(mrows)) for j in range(n)] for i in range(n)]
    cd = [C[i][i] if C[i][i] > 0 else 1.0 for i in range(n)]
    e = [[C[i][j] / math.sqrt(cd[i] * cd[j]) if (pat[i][j] and i != j) else 0.0 for j in range(n)] for i in range(n)]
    deg = [sum(1 for j in range(n) if pat[i][j] and j != i) for i in range(n)]
    wdeg = [sum(abs(e[i][j]) for j in range(n)) for i in range(n)]
    logc = [math.log(cd[i]) for i in range(n)]
    mean_log = sum(logc) / n
    dmax = max(max(deg), 1)
    h = [[logc[i] - mean_log, deg[i] / dmax] for i in range(n)]
    hs = [h]
    for layer in range(4):
        W1, W2, bb = params[f"W1_{layer}"], params[f"W2_{layer}"], params[f"b_{layer}"]
        fin, width = len(W1), len(W1[0])
        nb = [[sum(e[i][j] * h[j][f] for j in range(n)) for f in range(fin)] for i in range(n)]
        z = [[sum(h[i][f] * W1[f][o] for f in range(fin)) + sum(nb[i][f] * W2[f][o] for f in range(fin)) + bb[o]
              for o in range(width)] for i in range(n)]
        h = [[max(v, 0.0) for v in row] for row in z]
        hs.append(h)
    width = len(h[0])
    u = [sum(h[i][f] * params["ws"][f] for f in range(width)) for i in range(n)]
    d = [math.log1p(math.exp(sum(h[i][f] * params["wd"][f] for f in range(width)) + float(params["bd"])))
         for i in range(n)]
    delta = [d[i] / cd[i] for i in range(n)]
    m = {}
    for i in range(n):
        for j in range(n):
            if not pat[i][j]:
                continue
            if i == j:
                m[(i, j)] = delta[i]
            else:
                s = math.tanh(u[i] + u[j] + float(params["we"]) * e[i][j] + float(params["bs"]))
                m[(i, j)] = 0.9 * s * min(delta[i], delta[j]) * abs(e[i][j]) / max(wdeg[i], wdeg[j])
    return hs, m


def _pin_case():
    A = wl.weighted_grid(3, 2, seed=11)  # 12 x 9, every column coupled to its neighbours
    Ad = A.to_scipy().toarray()
    rng = np.random.default_rng(42)
    p = {}
    for name, shp in G.param_shapes():
        p[name] = rng.standard_normal(shp) * (0.6 if len(shp) == 2 else 0.3)
    p["bd"] = np.array(0.4)
    p["we"] = np.array(1.3)
    p["bs"] = np.array(-0.2)
    return A, Ad, p


def test_forward_layers_and_heads_match_loops_over_the_definition():
    A, Ad, p = _pin_case()
    g = G.Graph(A.to_scipy())
    m, cache = G.forward(g, p, keep=True)
    hs, mref = _forward_by_loops(Ad.tolist(), {k: v.tolist() for k, v in p.items()})
    for layer in range(5):
        np.testing.assert_allclose(cache["h"][layer], np.array(hs[layer]), rtol=1e-12, atol=1e-13)
    for layer in range(1, 5):  # every layer has active and inactive units, so the relu matters
        z = cache["z"][layer - 1]
        assert (z > 0).any() and (z < 0).any()
    rows, cols = g.rows, g.indices
    assert len(mref) == m.size
    ref = np.array([mref[(int(i), int(j))] for i, j in zip(rows, cols)])
    np.testing.assert_allclose(m, ref, rtol=1e-12, atol=1e-15)
    assert np.abs(ref[g.offdiag]).min() > 0  # the edge head reaches every off-diagonal entry


def test_forward_pin_separates_plausible_slips():
    # each slip of the layer stack changes M by far more than the pin's tolerance
    A, Ad, p = _pin_case()
    g = G.Graph(A.to_scipy())
    _, mref = _forward_by_loops(Ad.tolist(), {k: v.tolist() for k, v in p.items()})
    ref = np.array([mref[(int(i), int(j))] for i, j in zip(g.rows, g.indices)])

    def far(m):
        return np.max(np.abs(m - ref) / np.abs(ref)) > 1e-6

    swapped = dict(p)
    for layer in range(4):
        swapped[f"W1_{layer}"], swapped[f"W2_{layer}"] = p[f"W2_{layer}"], p[f"W1_{layer}"]
    assert far(G.forward(g, swapped))
    nobias = dict(p)
    for layer in range(4):
        nobias[f"b_{layer}"] = np.zeros_like(p[f"b_{layer}"])
    assert far(G.forward(g, nobias))
    gc = G.Graph(A.to_scipy())
    gc.E = gc.C.copy()  # messages weighted by c_ij instead of the normalised e_ij
    assert far(G.forward(gc, p))


def test_bf16_weights_round_only_the_layer_weights():
    # the network's layer weights in bfloat16: W1_l, W2_l rounded to nearest
    # even (the pinned rounding of the oracle), biases and heads unchanged
    from oracle.phsvds_fp64 import round_bf16

    p = G.init_params(6)
    q = G.bf16_weights(p)
    for name in p:
        if name.startswith(("W1_", "W2_")):
            np.testing.assert_array_equal(q[name], round_bf16(p[name].astype(np.float32)).astype(np.float64))
            assert np.abs(q[name] - p[name]).max() <= 2.0 ** -8 * np.abs(p[name]).max()
        else:
            np.testing.assert_array_equal(q[name], p[name])
