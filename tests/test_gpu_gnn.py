"""GPU parity of the learned preconditioner: graph of C = A^T A, forward M
values and loss gradients against the FP64 oracle (oracle/gnn_fp64.py)."""
import numpy as np
import pytest

import oracle
from oracle import gnn_fp64 as G
from paper_1607_01404_gb300 import binding as B
from paper_1607_01404_gb300 import workloads as wl
from subspace import check_dense_vectors

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
    p["bs"] = np.array(0.7)
    for l in range(G.LAYERS):
        p[f"b_{l}"] = 0.1 * rng.standard_normal(G.WIDTH)
    th = G.flatten(p).astype(np.float32)
    # the network applies its layer weights in bfloat16
    return th, G.bf16_weights(G.unflatten(th.astype(np.float64)))


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
    lam, V = np.linalg.eigh(ref.C.toarray())
    for T0, X0, ps, ss in ((rng.standard_normal((n, 5)), rng.standard_normal((n, 3)), 0, 0),
                           (rng.standard_normal((n, 8)), np.hstack([V[:, :4], rng.standard_normal((n, 4))]), 4, 30)):
        th, p = _theta(2)
        L, grad = g.loss_grad(th, T0, X0, ps, ss)
        Lr, gr = G.loss_and_grad(ref, p, T0, X0, ps, ss)
        gr = G.flatten(gr)
        assert abs(L - Lr) < 1e-4 * max(1.0, abs(Lr)), (L, Lr)
        err = np.linalg.norm(grad - gr) / np.linalg.norm(gr)
        assert err < G_TOL, (name, ps, ss, err)
    g.close()


def test_gradient_is_a_descent_direction_and_adam_steps():
    A = wl.weighted_grid(16, 2, seed=1)
    g = _gnn(A)
    rng = np.random.default_rng(5)
    T0, X0 = rng.standard_normal((g.n, 8)), rng.standard_normal((g.n, 8))
    th, p = _theta(4)
    L0, grad = g.loss_grad(th, T0, X0)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    th1 = th.copy()
    g.adam(th1, grad, m, v, 1, 1e-3)
    # first Adam step: m = 0.1 g, v = 0.001 g^2, update = lr * sign-like ratio
    mh = (0.1 * grad) / 0.1
    vh = (0.001 * grad * grad) / 0.001
    ref = th.astype(np.float64) - 1e-3 * mh / (np.sqrt(vh) + 1e-8)
    np.testing.assert_allclose(th1, ref, rtol=1e-5, atol=1e-7)
    # with the samples of th held fixed the loss decreases along the step
    gref = G.Graph(A.to_scipy())
    T, X = G.samples(gref, G.forward(gref, p), T0, X0, 4, 30)
    assert G.loss_fixed_samples(gref, G.bf16_weights(G.unflatten(th1.astype(np.float64))), T, X) < L0
    g.close()


def test_rejects_bad_arguments():
    A = wl.weighted_grid(6, 2, seed=1)
    g = _gnn(A)
    th, _ = _theta(0)
    R = np.ones((g.n, 9))
    with pytest.raises(B.SvdsError):
        g.loss_grad(th, R, R[:, :2])  # at most 8 columns per block
    Z = np.zeros((g.n, 2))
    with pytest.raises(B.SvdsError) as e:
        g.loss_grad(th, Z, np.ones((g.n, 2)))  # Rayleigh quotient 0 / 0
    assert e.value.code == B.SVDS_ERR_NUMERIC
    with pytest.raises(ValueError):
        g.forward(th[:-1])
    g.close()


def test_pairs_and_c_apply_match_the_graph():
    A = wl.weighted_grid(18, 2, seed=4)
    g = _gnn(A)
    ref = G.Graph(A.to_scipy())
    C = ref.C
    normC = abs(C).sum(axis=1).max()
    rq = []
    for s in (0, 4, 32):
        R, T = g.pairs(5, s, 9)
        assert np.linalg.norm(R - C @ T) <= 1e-13 * normC * np.linalg.norm(T)
        # damped Jacobi smoothing leaves the low end of the spectrum of C
        rq.append(np.mean(np.sum(T * (C @ T), axis=0) / np.sum(T * T, axis=0)))
    assert rq[0] > rq[1] > rq[2]
    X = np.random.default_rng(2).standard_normal((g.n, 7))
    Y = g.apply_c(X)
    assert np.linalg.norm(Y - C @ X) <= 1e-13 * normC * np.linalg.norm(X)
    g.close()


def _dense_sigma(A, k):
    s = np.linalg.svd(A.to_scipy().toarray(), compute_uv=False)
    return np.sort(s)[:k]


LEARNED_FORMS = [
    dict(),  # GD+k, FP64-class
    dict(stage1_precision=B.SVDS_FP32),
    dict(method_stage1=B.SVDS_JDQMR, stage1_precision=B.SVDS_FP32),
    dict(method_stage1=B.SVDS_JDQMR, innerPrecision=B.SVDS_DF64),
    dict(method_stage1=B.SVDS_JDQMR, stage1_precision=B.SVDS_NATIVE_FP64),
]


@pytest.mark.parametrize("form", range(len(LEARNED_FORMS)))
def test_solver_with_learned_preconditioner_is_correct(form):
    A = wl.weighted_grid(24, 2, seed=12)
    k = 5
    th = B.gnn_init(0)
    r = B.svds(A, k, "smallest", tol=1e-10, maxBlockSize=2, precond=B.SVDS_PRECOND_LEARNED, precondParams=th,
               **LEARNED_FORMS[form])
    assert r["nconv"] == k
    sd = _dense_sigma(A, k)
    np.testing.assert_allclose(r["sigma"], sd, rtol=1e-10)
    normA = np.linalg.svd(A.to_scipy().toarray(), compute_uv=False).max()
    res = oracle.triplet_residuals(A, r["sigma"], r["U"], r["V"])
    assert res.max() <= 1e-10 * normA * 1.0000001
    check_dense_vectors(A, r)
    assert r["stats"]["seconds_precond"] > 0


def test_learned_preconditioner_from_model_file_and_largest_ignores_it(tmp_path):
    A = wl.weighted_grid(16, 2, seed=3)
    th = B.gnn_init(5)
    p = tmp_path / "m.bin"
    B.gnn_save(p, th)
    r1 = B.svds(A, 3, "smallest", tol=1e-9, precond=B.SVDS_PRECOND_LEARNED, precondModel=str(p))
    r2 = B.svds(A, 3, "smallest", tol=1e-9, precond=B.SVDS_PRECOND_LEARNED, precondParams=th)
    np.testing.assert_array_equal(r1["sigma"], r2["sigma"])
    r3 = B.svds(A, 3, "largest", tol=1e-9, precond=B.SVDS_PRECOND_LEARNED, precondParams=th)
    assert r3["stats"]["seconds_precond"] == 0
    np.testing.assert_allclose(r3["sigma"], np.sort(np.linalg.svd(A.to_scipy().toarray(), compute_uv=False))[::-1][:3],
                               rtol=1e-10)


def test_short_training_lowers_the_loss():
    from paper_1607_01404_gb300 import gnn_train

    theta, hist = gnn_train.train("wgrid2d", 20, seeds=range(3), epochs=12, lr=3e-3)
    assert np.all(np.isfinite(theta))
    assert hist[-1] < hist[0]


@pytest.mark.parametrize("family,N,model", [("wgrid2d", 128, "wgrid2d.bin"), ("wgrid3d", 40, "wgrid3d.bin")])
def test_trained_models_gain_over_jacobi(family, N, model):
    """The committed trained networks on a held-out seed: fewer products with A
    (deterministic counts) than the Jacobi solver, the same triplets."""
    import os

    from paper_1607_01404_gb300 import gnn_train

    A = gnn_train.training_matrix(family, N, 10042)
    path = os.path.join(os.path.dirname(B.__file__), "gnn_models", model)
    out = {}
    for name, kw in (("jacobi", dict(precond=B.SVDS_PRECOND_JACOBI)),
                     ("learned", dict(precond=B.SVDS_PRECOND_LEARNED, precondModel=path))):
        r = B.svds(A, 8, "smallest", tol=1e-10, maxBlockSize=4, stage1_precision=B.SVDS_FP32, **kw)
        assert r["nconv"] == 8
        out[name] = r
    mv = {k: v["stats"]["matvecs_stage1"] + v["stats"]["matvecs_stage2"] for k, v in out.items()}
    assert out["learned"]["stats"]["precond_fallback"] == 0
    assert mv["learned"] < 0.85 * mv["jacobi"], mv
    # both runs meet ||r|| <= 1e-10 ||A||; the values agree to 1e-10 (quadratic in ||r||)
    np.testing.assert_allclose(out["learned"]["sigma"], out["jacobi"]["sigma"], rtol=1e-10)


def _fallback_case():
    A = wl.weighted_grid(24, 2, seed=10002)
    kw = dict(maxBlockSize=2, stage1_precision=B.SVDS_FP32, method_stage1=B.SVDS_JDQMR, maxMatvecs=2000000)
    ref = B.svds(A, 4, "smallest", 1e-10, precond=B.SVDS_PRECOND_JACOBI, **kw)
    assert ref["nconv"] == 4 and ref["stats"]["precond_fallback"] == 0
    return A, kw, ref


@pytest.mark.parametrize("bad", ["underflow", "nan"])
def test_learned_preconditioner_rejected_falls_back_to_jacobi(bad):
    """An unusable M (a diagonal that underflows to zero: zero weights and a
    node-head bias of -200; or a NaN node-head bias, which reaches M's
    diagonal: a NaN in a layer weight would be cleared by the ReLU) is
    replaced by the Jacobi preconditioner before the first iteration, with
    the same triplets."""
    A, kw, ref = _fallback_case()
    th = np.zeros(B.gnn_num_params(), dtype=np.float32)
    if bad == "underflow":
        th[-1] = -200.0  # bd: softplus(-200) is 0 in FP32
    else:
        th[:] = B.gnn_init(0)
        th[-1] = np.nan  # bd
    r = B.svds(A, 4, "smallest", 1e-10, precond=B.SVDS_PRECOND_LEARNED, precondParams=th, **kw)
    assert r["nconv"] == 4
    assert r["stats"]["precond_fallback"] == 1
    np.testing.assert_allclose(r["sigma"], ref["sigma"], rtol=1e-10)
    check_dense_vectors(A, r)


def test_learned_preconditioner_stall_falls_back_to_jacobi():
    """A poor M (node-head weights that spread the diagonal over many orders of
    magnitude) in GD+k with a one-iteration stall window: the residual fails to
    reach a new minimum at some outer iteration, Jacobi takes over, and the
    triplets are the Jacobi run's."""
    A, kw, ref = _fallback_case()
    kw = dict(kw, method_stage1=B.SVDS_GDPK)  # GD+k: many outer iterations, small steps
    th = B.gnn_init(3)
    rng = np.random.default_rng(5)
    n = G.n_params()
    th[n - 3 - G.WIDTH:n - 3] = (8.0 * rng.standard_normal(G.WIDTH)).astype(np.float32)  # wd (node head)
    r = B.svds(A, 4, "smallest", 1e-10, precond=B.SVDS_PRECOND_LEARNED, precondParams=th, precondStallIts=1, **kw)
    assert r["nconv"] == 4
    assert r["stats"]["precond_fallback"] == 2
    np.testing.assert_allclose(r["sigma"], ref["sigma"], rtol=1e-10)
    check_dense_vectors(A, r)
