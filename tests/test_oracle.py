"""Pins of the CPU oracle against closed forms, dense LAPACK and invariants.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
swapped half of B, a wrong sign in the lower bound, a transposed operand) fails.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import phsvds_fp64 as O
from paper_1607_01404_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))


def _grid_sigma(N, dims):
    t = 4.0 * np.sin(np.arange(1, N + 1) * np.pi / (2 * (N + 1))) ** 2
    if dims == 2:
        s = t[:, None] + t[None, :]
    else:
        s = t[:, None, None] + t[None, :, None] + t[None, None, :]
    return np.sort(np.sqrt(s.ravel()))


def _golden_grid2d():
    vals = [float(l) for l in open(os.path.join(HERE, "golden", "grid2d_N32_sigma.txt")) if not l.startswith("#")]
    return np.array(vals[:5]), np.array(vals[5:])


# ---------------------------------------------------------------- operators
def test_spmm_definition():
    A = wl.random_illconditioned(60, 25, 16, seed=3)
    X = wl.dense_block(25, 3, seed=1)
    D = A.to_scipy().toarray()
    ref = np.array([[sum(D[i, j] * X[j, c] for j in range(25)) for c in range(3)] for i in range(60)])
    np.testing.assert_allclose(oracle.spmm(A, X), ref, rtol=0, atol=1e-13)
    Y = wl.dense_block(60, 2, seed=2)
    np.testing.assert_allclose(oracle.spmm_t(A, Y), D.T @ Y, rtol=0, atol=1e-13)


def test_apply_B_matches_dense_augmented_matrix():
    A = wl.random_illconditioned(40, 15, 8, seed=1)
    D = A.to_scipy().toarray()
    m, n = D.shape
    B = np.zeros((m + n, m + n))
    B[:n, n:] = D.T  # [0 A^T; A 0] acting on [v; u]
    B[n:, :n] = D
    X = wl.dense_block(m + n, 3, seed=4)
    np.testing.assert_allclose(oracle.apply_B(A, X), B @ X, atol=1e-13)
    np.testing.assert_allclose(oracle.apply_C(A, X[:n]), D.T @ D @ X[:n], atol=1e-12)


def test_B_spectrum_is_pm_sigma_and_zeros():
    # Eq. 2.5: eigenvalues of B are +-sigma_i and m - n zeros
    A = wl.random_illconditioned(30, 12, 6, seed=7)
    D = A.to_scipy().toarray()
    m, n = D.shape
    cols = np.column_stack([oracle.apply_B(A, e[:, None]).ravel() for e in np.eye(m + n)])
    ev = np.sort(np.linalg.eigvalsh(cols))
    s = np.linalg.svd(D, compute_uv=False)
    ref = np.sort(np.concatenate([s, -s, np.zeros(m - n)]))
    np.testing.assert_allclose(ev, ref, atol=1e-12)


def test_triplet_residual_definition():
    A = wl.random_illconditioned(50, 20, 8, seed=2)
    D = A.to_scipy().toarray()
    U, s, Vt = np.linalg.svd(D, full_matrices=False)
    r = oracle.triplet_residuals(A, s[:3], U[:, :3], Vt[:3].T)
    assert r.max() < 1e-13
    # perturbed triplet: compare against the formula evaluated with dense algebra
    rng = np.random.default_rng(0)
    u = U[:, 0] + 1e-3 * rng.standard_normal(50)
    v = Vt[0] + 1e-3 * rng.standard_normal(20)
    sg = s[0] * (1 + 1e-4)
    ref = math.sqrt(np.sum((D @ v - sg * u) ** 2) + np.sum((D.T @ u - sg * v) ** 2))
    got = oracle.triplet_residuals(A, np.array([sg]), u[:, None], v[:, None])[0]
    assert abs(got - ref) <= 1e-14 * ref
    # each half matters (a dropped term would fail one of these)
    only_left = math.sqrt(np.sum((D @ v - sg * u) ** 2))
    assert got > 1.05 * only_left


# ----------------------------------------------------------- orthonormalise
def test_orthonormalize_against_basis():
    rng = np.random.default_rng(1)
    V, _ = np.linalg.qr(rng.standard_normal((200, 7)))
    T = rng.standard_normal((200, 4))
    Q = oracle.orthonormalize(T, V)
    assert np.abs(Q.T @ Q - np.eye(4)).max() < 1e-14
    assert np.abs(V.T @ Q).max() < 1e-14
    # span(Q) lies in span([V T])
    P = np.hstack([V, T])
    coef, *_ = np.linalg.lstsq(P, Q, rcond=None)
    assert np.abs(P @ coef - Q).max() < 1e-12


def test_orthonormalize_breakdown_replaces_dependent_columns():
    rng = np.random.default_rng(2)
    V, _ = np.linalg.qr(rng.standard_normal((100, 5)))
    T = np.hstack([V[:, :1] * 3.0, rng.standard_normal((100, 1))])  # first column lies in span(V)
    T = np.hstack([T, T[:, 1:2]])  # duplicated column
    Q = oracle.orthonormalize(T, V)
    assert Q.shape[1] == 3
    assert np.abs(Q.T @ Q - np.eye(3)).max() < 1e-13
    assert np.abs(V.T @ Q).max() < 1e-13


def test_norm_estimate():
    A = wl.grid_difference(32, 2)
    s = _grid_sigma(32, 2)
    # Lanczos approaches ||A|| from below; a 1e-4 relative shortfall only
    # tightens the tolerance ||A|| delta by the same factor
    est = oracle.estimate_norm(A)
    assert s[-1] * (1 - 1e-4) < est <= s[-1] * (1 + 1e-12)
    R = wl.random_illconditioned(300, 100, 16, seed=3)
    s2 = np.linalg.svd(R.to_scipy().toarray(), compute_uv=False)
    est = oracle.estimate_norm(R)
    assert est <= s2[0] * (1 + 1e-12) and est > s2[0] * (1 - 1e-4)


# --------------------------------------------------------------- Algorithm 1
def _angle_to_span(x, basis):
    """sin of the angle between x and span(basis) (basis orthonormal)."""
    x = x / np.linalg.norm(x)
    return np.linalg.norm(x - basis @ (basis.T @ x))


def _grid2d_singular_subspace(N, sigma, tol=1e-9):
    """Exact right singular vectors of the 2D grid operator for the value sigma:
    Kronecker products of s_i(t) = sin(i t pi / (N+1)) (D^T D = tridiag(-1,2,-1))."""
    t = np.arange(1, N + 1)
    lam = 4.0 * np.sin(t * np.pi / (2 * (N + 1))) ** 2
    vecs = []
    for i in range(N):
        for j in range(N):
            if abs(math.sqrt(lam[i] + lam[j]) - sigma) < tol:
                si = np.sin((i + 1) * t * np.pi / (N + 1))
                sj = np.sin((j + 1) * t * np.pi / (N + 1))
                vecs.append(np.kron(si, sj))
    Q, _ = np.linalg.qr(np.array(vecs).T)
    return Q


@pytest.mark.parametrize("target", ["smallest", "largest"])
def test_phsvds_grid2d_closed_form(target):
    A = wl.grid_difference(32, 2)
    small, large = _golden_grid2d()
    normA = large[0]
    r = oracle.phsvds(A, 5, target, 1e-10, b=1, V0=wl.start_block(A.n, 1, 0), normA=normA)
    ex = small if target == "smallest" else large
    np.testing.assert_allclose(r["sigma"], ex, rtol=1e-10)
    assert r["rnorm"].max() <= 1e-10 * normA
    for j in range(5):
        Q = _grid2d_singular_subspace(32, ex[j])
        assert _angle_to_span(r["V"][:, j], Q) < 1e-8
    # orthonormal columns
    assert np.abs(r["V"].T @ r["V"] - np.eye(5)).max() < 1e-10
    assert np.abs(r["U"].T @ r["U"] - np.eye(5)).max() < 1e-10


@pytest.mark.parametrize("target", ["smallest", "largest"])
def test_phsvds_stage2_grid2d(target):
    """Stage 1 stopped at an FP32-level floor, so stage 2 on B must refine."""
    A = wl.grid_difference(32, 2)
    small, large = _golden_grid2d()
    normA = large[0]
    r = oracle.phsvds(A, 5, target, 1e-10, b=2, V0=wl.start_block(A.n, 2, 0), normA=normA,
                      u_stage1=2.0 ** -24, polish=False)
    assert r["stage2_used"]
    ex = small if target == "smallest" else large
    np.testing.assert_allclose(r["sigma"], ex, rtol=1e-10)
    assert r["rnorm"].max() <= 1e-10 * normA
    if target == "smallest":
        # Sec. 3.1: sigma_i in [s_i - sqrt(2) ||r^C_i|| / s_i, s_i] for the stage-1 values
        s1, rC = r["sigma1"], r["rC"]
        lower = s1 - math.sqrt(2.0) * rC / s1
        assert np.all(lower <= ex * (1 + 1e-12))
        assert np.all(s1 >= ex * (1 - 1e-12))


@pytest.mark.parametrize("target,tol,u1", [("smallest", 1e-10, O.EPS), ("largest", 1e-10, O.EPS),
                                           ("smallest", 1e-13, O.EPS), ("largest", 1e-10, 2.0 ** -24),
                                           ("smallest", 1e-10, 2.0 ** -24)])
def test_phsvds_random_vs_lapack(target, tol, u1):
    A = wl.random_illconditioned(600, 200, 16, seed=11)
    D = A.to_scipy().toarray()
    U, s, Vt = np.linalg.svd(D, full_matrices=False)
    k, b = 4, 2
    r = oracle.phsvds(A, k, target, tol, b=b, V0=wl.start_block(A.n, b, 1), u_stage1=u1)
    idx = np.arange(k) if target == "largest" else np.arange(len(s) - 1, len(s) - 1 - k, -1)
    np.testing.assert_allclose(r["sigma"], s[idx], rtol=1e-10)
    normA = s[0]
    assert r["rnorm"].max() <= tol * normA
    for j, i in enumerate(idx):
        # sin(angle) <= ||r|| / gap for a separated singular value
        gap = min(abs(s[i] - s[i2]) for i2 in range(len(s)) if i2 != i)
        bound = 2 * r["rnorm"][j] / gap + 1e-12
        assert _angle_to_span(r["V"][:, j], Vt[i][:, None]) <= bound
        assert _angle_to_span(r["U"][:, j], U[:, i][:, None]) <= bound
        if gap > 1e-2 * normA:
            assert _angle_to_span(r["V"][:, j], Vt[i][:, None]) < 1e-8
    if tol < 1e-12 and target == "smallest":
        # the FP64 stage-1 floor 10 eps ||C|| exceeds sqrt(l ||C||) delta here
        assert r["stage2_used"]


def test_phsvds_wide_matrix_uses_transpose():
    A = wl.random_illconditioned(300, 120, 16, seed=5)
    At = A.to_scipy().T.tocsr()  # 120 x 300, m < n
    s = np.linalg.svd(At.toarray(), compute_uv=False)
    r = oracle.phsvds(At, 3, "largest", 1e-10, b=1)
    np.testing.assert_allclose(r["sigma"], s[:3], rtol=1e-10)
    assert r["U"].shape == (120, 3) and r["V"].shape == (300, 3)
    assert oracle.triplet_residuals(At, r["sigma"], r["U"], r["V"]).max() <= 1e-10 * s[0]


def test_phsvds_grid3d_small_closed_form():
    A = wl.grid_difference(7, 3)  # 1176 x 343
    s = _grid_sigma(7, 3)
    r = oracle.phsvds(A, 4, "smallest", 1e-10, b=4, V0=wl.start_block(A.n, 4, 2), normA=s[-1])
    np.testing.assert_allclose(r["sigma"], s[:4], rtol=1e-10)
    assert r["rnorm"].max() <= 1e-10 * s[-1]


def test_value_error_bound_eq_2_1():
    # Eq. 2.1: a stage-1 value with ||C v - l v|| <= ||A||^2 eps has relative
    # error <= kappa_i^2 eps; check on the oracle's stage-1 output (stage 2 off).
    A = wl.random_illconditioned(400, 100, 16, seed=8)
    s = np.linalg.svd(A.to_scipy().toarray(), compute_uv=False)
    r = oracle.phsvds(A, 3, "smallest", 1e-14, b=3, stage2=False, V0=wl.start_block(A.n, 3, 3))
    kappa = s[0] / s[::-1][:3]
    rel = np.abs(r["sigma1"] - s[::-1][:3]) / s[::-1][:3]
    assert np.all(rel <= 10 * O.FLOOR_C * kappa ** 2 * O.EPS + 1e-13)


def test_round_bf16_definition():
    """Round to nearest even on the 8-bit significand of bfloat16."""
    from oracle.phsvds_fp64 import round_bf16

    e = 2.0 ** -7  # spacing of bfloat16 numbers in [1, 2)
    x = np.array([1.0, -2.5, 0.15625, 1 + e / 2, 1 + 3 * e / 2, 1 + e / 2 + 2.0 ** -20, -(1 + e / 2 + 2.0 ** -20),
                  3.0e-39, 0.0], dtype=np.float64)
    want = np.array([1.0, -2.5, 0.15625, 1.0, 1 + 2 * e, 1 + e, -(1 + e), None, 0.0], dtype=object)
    got = round_bf16(x.astype(np.float32)).astype(np.float64)
    for g, w in zip(got[:7], want[:7]):
        assert g == w
    assert got[8] == 0.0
    # every result is a bfloat16 number, within half a spacing (at most 2^-8 relative)
    rng = np.random.default_rng(0)
    v = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-3, 3, 20000)).astype(np.float32)
    r = round_bf16(v)
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)
    assert np.all(np.abs(r.astype(np.float64) - v) <= 2.0 ** -8 * np.abs(v.astype(np.float64)))
    # monotone
    s = np.sort(v)
    assert np.all(np.diff(round_bf16(s).astype(np.float64)) >= 0)


def test_jd_correction_exact_definition():
    """Diagonal C and x = e_0: t = (C - eta)^-1 b on the other coordinates; in
    general the projected equation holds and t is orthogonal to x."""
    from oracle.phsvds_fp64 import jd_correction_exact

    d = np.array([1.0, 2.0, 3.5, 5.0, 7.0])
    C = np.diag(d)
    X = np.eye(5)[:, :1]
    b = np.array([[0.0], [1.0], [-2.0], [0.5], [3.0]])
    t = jd_correction_exact(C, X, b, np.array([2.5]))
    want = np.zeros(5)
    want[1:] = b[1:, 0] / (d[1:] - 2.5)
    np.testing.assert_allclose(t[:, 0], want, rtol=1e-13, atol=1e-15)
    rng = np.random.default_rng(2)
    M = rng.standard_normal((30, 30))
    C = M @ M.T
    X = np.linalg.qr(rng.standard_normal((30, 2)))[0]
    B = rng.standard_normal((30, 2))
    B -= X * np.sum(X * B, axis=0)
    eta = np.array([1.3, 7.7])
    T = jd_correction_exact(C, X, B, eta)
    for j in range(2):
        P = np.eye(30) - np.outer(X[:, j], X[:, j])
        np.testing.assert_allclose(P @ (C - eta[j] * np.eye(30)) @ P @ T[:, j], B[:, j], atol=1e-10 * np.abs(B).max())
        assert abs(X[:, j] @ T[:, j]) < 1e-12 * np.linalg.norm(T[:, j])


def test_condest_bounds_and_limit():
    """Condition-number estimate (Sec. 5): Ritz values lie inside the spectrum,
    so the estimate never exceeds kappa; with ||r^C|| <= 0.1 lambda at both ends
    (and convergence to the extremes) it is within sqrt(1.1 / 0.9) of kappa;
    as rel_tol -> 0 it reduces to the exact kappa of a dense SVD."""
    for A in (wl.grid_difference(12, 3).to_scipy(), wl.random_illconditioned(900, 300, 16, seed=4).to_scipy()):
        s = np.linalg.svd(A.toarray(), compute_uv=False)
        kappa = s[0] / s[-1]
        r = O.condest(A, 0.1)
        assert r["sigma_max"] <= s[0] * (1 + 1e-12) and r["sigma_min"] >= s[-1] * (1 - 1e-12)
        assert kappa * math.sqrt(0.9 / 1.1) <= r["kappa"] <= kappa * (1 + 1e-12), (r["kappa"], kappa)
        assert r["rC_max"] <= 0.1 * r["sigma_max"] ** 2 * (1 + 1e-12)
        assert r["rC_min"] <= 0.1 * r["sigma_min"] ** 2 * (1 + 1e-12)
        tight = O.condest(A, 1e-12)
        assert abs(tight["kappa"] / kappa - 1) < 1e-9, (tight["kappa"], kappa)


def test_condest_wide_matrix_and_no_preconditioner():
    A = wl.random_illconditioned(700, 250, 16, seed=8).to_scipy()
    s = np.linalg.svd(A.toarray(), compute_uv=False)
    r = O.condest(A.T.tocsr(), 1e-12, precond="none")  # 250 x 700: works on (A^T)^T = A
    assert abs(r["kappa"] * s[-1] / s[0] - 1) < 1e-9


def test_block_jacobi_definition():
    """Block Jacobi on A^T A: bs = 1 is Jacobi; a single block is the inverse
    of (shifted) C; every diagonal block of M C is the identity up to the shift;
    M is symmetric positive definite; an empty column gets the entry 1."""
    A = wl.random_illconditioned(400, 90, 8, seed=6).to_scipy().tolil()
    A[:, 17] = 0.0  # an empty column
    A = A.tocsr()
    C = (A.T @ A).toarray()
    d = np.diag(C)
    M1 = O.block_jacobi(A, 1).toarray()
    # one column per block: delta = 1e-10 c_ii, and 1 for the empty column
    np.testing.assert_allclose(np.diag(M1), np.where(d > 0, 1.0 / (np.where(d > 0, d, 1.0) * (1 + 1e-10)), 1.0),
                               rtol=1e-14)
    assert np.count_nonzero(M1 - np.diag(np.diag(M1))) == 0
    Mall = O.block_jacobi(A, 90).toarray()
    Cs = C.copy()
    Cs[17, 17] = 1.0
    Cs += 1e-10 * d.max() * np.eye(90)
    np.testing.assert_allclose(Mall @ Cs, np.eye(90), atol=1e-9)
    for bs in (7, 32):
        M = O.block_jacobi(A, bs).toarray()
        np.testing.assert_allclose(M, M.T, atol=0)
        assert np.linalg.eigvalsh(M).min() > 0
        for g0 in range(0, 90, bs):
            I = slice(g0, min(90, g0 + bs))
            CII = C[I, I].copy()
            dI = np.diag(CII).copy()
            delta = 1e-10 * dI.max()
            dI[dI == 0] = 1.0
            np.fill_diagonal(CII, dI + delta)
            np.testing.assert_allclose(M[I, I] @ CII, np.eye(CII.shape[0]), atol=1e-9)
            if g0 + bs < 90:
                assert np.all(M[I, g0 + bs:] == 0)
            if g0 <= 17 < g0 + bs:
                # the empty column decouples: its entry is 1 / (1 + delta_I)
                assert abs(M[17, 17] - 1.0 / (1.0 + delta)) < 1e-12


def test_phsvds_block_jacobi_preconditioner_closed_form():
    A = wl.grid_difference(8, 3)
    t = 4.0 * np.sin(np.arange(1, 9) * np.pi / 18) ** 2
    s = np.sort(np.sqrt((t[:, None, None] + t[None, :, None] + t[None, None, :]).ravel()))
    r = O.phsvds(A.to_scipy(), 3, "smallest", 1e-10, b=2, precond="block_jacobi", bj_block=16)
    np.testing.assert_allclose(r["sigma"], s[:3], rtol=1e-10)


def test_subspace_helper_accepts_oracle_vectors_and_rejects_wrong_ones():
    """The angle checks of the GPU tests (tests/subspace.py) on oracle results:
    the closed-form and dense subspaces accept the oracle's vectors (config 1,
    whose 5th smallest value is a double value cut at k = 5), and reject a
    vector taken from another value's subspace."""
    import pytest as _pt

    from subspace import check_dense_vectors, check_grid_vectors

    A = wl.grid_difference(32, 2)
    small, large = _golden_grid2d()
    r = oracle.phsvds(A, 5, "smallest", 1e-10, b=1, V0=wl.start_block(A.n, 1, 0), normA=large[0])
    assert check_grid_vectors(A, 32, 2, r) < 1e-8
    bad = dict(r, V=r["V"][:, [1, 0, 2, 3, 4]])
    with _pt.raises(AssertionError):
        check_grid_vectors(A, 32, 2, bad)
    R = wl.random_illconditioned(600, 200, 16, seed=11)
    rr = oracle.phsvds(R, 3, "largest", 1e-10, b=1)
    assert check_dense_vectors(R, rr) < 1e-8
    with _pt.raises(AssertionError):
        check_dense_vectors(R, dict(rr, U=rr["U"][:, [0, 2, 1]]))
