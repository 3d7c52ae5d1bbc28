"""End-to-end parity: triplets from the CUDA path (through the C-ABI) against
the oracle, closed forms and certificates recomputed on the host in FP64.

Bars (from the method's accuracy statement): relative singular-value error
<= 1e-10, triplet residual of Eq. (res) <= tol ||A|| recomputed in FP64 from
the returned vectors, sin(angle) to the exact singular subspace <= 1e-8 for
values separated by more than 1e-2 ||A||, else <= ||r|| / gap.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import phsvds_fp64 as O
from paper_1607_01404_gb300 import binding as B
from paper_1607_01404_gb300 import build as BLD
from paper_1607_01404_gb300 import workloads as wl
from subspace import check_dense_vectors, check_grid_vectors

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    BLD.build()
    B.lib()


def _grid_sigma(N, dims):
    t = 4.0 * np.sin(np.arange(1, N + 1) * np.pi / (2 * (N + 1))) ** 2
    s = t[:, None] + t[None, :] if dims == 2 else t[:, None, None] + t[None, :, None] + t[None, None, :]
    return np.sort(np.sqrt(s.ravel()))


def _sin_angle(x, basis):
    x = x / np.linalg.norm(x)
    return np.linalg.norm(x - basis @ (basis.T @ x))


def _check_certificate(A, r, tol, normA, k):
    assert r["nconv"] == k, r
    res = oracle.triplet_residuals(A, r["sigma"], r["U"], r["V"])
    assert res.max() <= tol * normA * 1.0000001, res / normA
    # the library evaluates Eq. (res) in double-float (unit 2^-48): agreement up to
    # a few units of 2^-48 ||A|| absolute
    np.testing.assert_allclose(r["rnorm"], res, rtol=1e-3, atol=16 * 2.0 ** -48 * normA)
    assert np.abs(r["V"].T @ r["V"] - np.eye(k)).max() < 1e-8
    assert np.abs(r["U"].T @ r["U"] - np.eye(k)).max() < 1e-8


def _compare_to_dense(A, r, target, k, tol):
    D = A.to_scipy().toarray()
    U, s, Vt = np.linalg.svd(D, full_matrices=False)
    idx = np.arange(k) if target == "largest" else np.arange(len(s) - 1, len(s) - 1 - k, -1)
    np.testing.assert_allclose(r["sigma"], s[idx], rtol=1e-10)
    _check_certificate(A, r, tol, s[0], k)
    for j, i in enumerate(idx):
        gap = min(abs(s[i] - s[i2]) for i2 in range(len(s)) if i2 != i)
        bound = 2 * tol * s[0] / gap + 1e-12
        if gap > 1e-2 * s[0]:
            bound = min(bound, 1e-8)
        assert _sin_angle(r["V"][:, j], Vt[i][:, None]) <= bound
        assert _sin_angle(r["U"][:, j], U[:, i][:, None]) <= bound


@pytest.mark.parametrize("target", ["smallest", "largest"])
def test_grid2d_closed_form_and_oracle(target):
    A = wl.grid_difference(32, 2)
    s = _grid_sigma(32, 2)
    ex = s[:5] if target == "smallest" else s[::-1][:5]
    r = B.svds(A, 5, target, 1e-10, maxBlockSize=1, initV=wl.start_block(A.n, 1, 0), maxMatvecs=200000)
    o = oracle.phsvds(A, 5, target, 1e-10, b=1, V0=wl.start_block(A.n, 1, 0))
    np.testing.assert_allclose(r["sigma"], ex, rtol=1e-10)
    np.testing.assert_allclose(r["sigma"], o["sigma"], rtol=1e-10)
    _check_certificate(A, r, 1e-10, s[-1], 5)
    # vectors: each in the closed-form subspace of its value (the 5th value is
    # double and cut at k = 5, so its vector may be any unit vector of that plane)
    check_grid_vectors(A, 32, 2, r)
    # the ||A|| estimate is a Lanczos lower bound within a few 1e-3 (clustered
    # top; the steps stop once the top Ritz value moves by <= 1e-3 relative)
    assert s[-1] * (1 - 1e-2) <= r["stats"]["aNorm"] <= s[-1] * (1 + 1e-12)


@pytest.mark.parametrize("target", ["smallest", "largest"])
@pytest.mark.parametrize("b", [1, 2, 4])
def test_random_vs_dense_and_oracle(target, b):
    A = wl.random_illconditioned(1500, 500, 16, seed=11)
    k = 4
    r = B.svds(A, k, target, 1e-10, maxBlockSize=b, initV=wl.start_block(A.n, b, 1), maxMatvecs=400000)
    _compare_to_dense(A, r, target, k, 1e-10)
    o = oracle.phsvds(A, k, target, 1e-10, b=b, V0=wl.start_block(A.n, b, 1))
    np.testing.assert_allclose(r["sigma"], o["sigma"], rtol=1e-10)


@pytest.mark.parametrize("target", ["smallest", "largest"])
def test_stage2_tight_tolerance(target):
    """tol 1e-13: the FP64-class stage-1 floor exceeds the smallest values' bound,
    so stage 2 on B (refined extraction for the smallest) must finish the job."""
    A = wl.random_illconditioned(900, 300, 16, seed=13)
    r = B.svds(A, 3, target, 1e-13, maxBlockSize=2, initV=wl.start_block(A.n, 2, 2), maxMatvecs=600000)
    _compare_to_dense(A, r, target, 3, 1e-13)
    if target == "smallest":
        assert r["stats"]["stage2_used"] == 1


@pytest.mark.parametrize("target", ["smallest", "largest"])
@pytest.mark.parametrize("polish", [1, 0])
def test_mixed_precision_stage1(target, polish):
    A = wl.grid_difference(24, 2)
    s = _grid_sigma(24, 2)
    ex = s[:4] if target == "smallest" else s[::-1][:4]
    r = B.svds(A, 4, target, 1e-10, maxBlockSize=2, stage1_precision=B.SVDS_FP32, stage1_polish=polish,
               initV=wl.start_block(A.n, 2, 3), maxMatvecs=400000)
    np.testing.assert_allclose(r["sigma"], ex, rtol=1e-10)
    _check_certificate(A, r, 1e-10, s[-1], 4)
    check_grid_vectors(A, 24, 2, r)
    assert r["stats"]["matvecs_stage1_lowprec"] > 0
    if not polish:
        assert r["stats"]["stage2_used"] == 1


def test_native_fp64_mode():
    A = wl.random_illconditioned(1200, 400, 16, seed=17)
    r = B.svds(A, 3, "smallest", 1e-10, maxBlockSize=2, stage1_precision=B.SVDS_NATIVE_FP64, maxMatvecs=400000)
    _compare_to_dense(A, r, "smallest", 3, 1e-10)


def test_wide_matrix():
    A = wl.random_illconditioned(700, 250, 16, seed=19)
    At = A.to_scipy().T.tocsr()
    At.sort_indices()
    W = wl.CSR(At.shape[0], At.shape[1], At.indptr.astype(np.int32), At.indices.astype(np.int32), At.data, "wide")
    r = B.svds(W, 3, "largest", 1e-10, maxBlockSize=1, maxMatvecs=200000)
    assert r["U"].shape == (250, 3) and r["V"].shape == (700, 3)
    _compare_to_dense(W, r, "largest", 3, 1e-10)


def test_grid3d_closed_form_block4():
    A = wl.grid_difference(10, 3)
    s = _grid_sigma(10, 3)
    r = B.svds(A, 4, "smallest", 1e-10, maxBlockSize=4, maxMatvecs=400000)
    np.testing.assert_allclose(r["sigma"], s[:4], rtol=1e-10)
    _check_certificate(A, r, 1e-10, s[-1], 4)
    check_grid_vectors(A, 10, 3, r)


def test_weighted_grid_vs_oracle_and_jacobi_none():
    A = wl.weighted_grid(20, 2, seed=10000)
    s = np.linalg.svd(A.to_scipy().toarray(), compute_uv=False)
    rj = B.svds(A, 4, "smallest", 1e-10, maxBlockSize=2, precond=B.SVDS_PRECOND_JACOBI, maxMatvecs=600000)
    rn = B.svds(A, 4, "smallest", 1e-10, maxBlockSize=2, precond=B.SVDS_PRECOND_NONE, maxMatvecs=600000)
    for r in (rj, rn):
        np.testing.assert_allclose(r["sigma"], s[::-1][:4], rtol=1e-10)
        _check_certificate(A, r, 1e-10, s[0], 4)
        check_dense_vectors(A, r)


def test_odd_block_k1_and_sign_convention():
    A = wl.random_illconditioned(800, 300, 16, seed=23)
    r = B.svds(A, 1, "largest", 1e-10, maxBlockSize=3, maxMatvecs=200000)
    _compare_to_dense(A, r, "largest", 1, 1e-10)
    v = r["V"][:, 0]
    assert v[np.argmax(np.abs(v))] > 0


def test_budget_exhausted_returns_maxit():
    A = wl.grid_difference(32, 2)
    r = B.svds(A, 5, "smallest", 1e-10, maxBlockSize=1, maxMatvecs=50)
    assert r["rc"] == B.SVDS_ERR_MAXIT
    assert r["nconv"] == 0


def test_device_csr_input_and_repeat_solves():
    A = wl.random_illconditioned(1000, 400, 16, seed=29)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(A.rowptr).to(dev)
    ci = torch.from_numpy(A.colidx).to(dev)
    va = torch.from_numpy(A.vals).to(dev)
    h = B.svds_create(rp, ci, va, A.m, A.n, B.make_opts(maxBlockSize=2, maxMatvecs=300000), on_device=True)
    try:
        s1 = B.svds_solve(h, 3, B.SVDS_LARGEST, 1e-10)
        s2 = B.svds_solve(h, 3, B.SVDS_LARGEST, 1e-10)
    finally:
        h.close()
    np.testing.assert_array_equal(s1[0], s2[0])  # deterministic
    D = A.to_scipy().toarray()
    np.testing.assert_allclose(s1[0], np.linalg.svd(D, compute_uv=False)[:3], rtol=1e-10)


def test_device_csr_validation():
    dev = torch.device("cuda:0")
    rp = torch.tensor([0, 2, 3], dtype=torch.int32, device=dev)
    ci = torch.tensor([1, 0, 1], dtype=torch.int32, device=dev)  # unsorted row 0
    va = torch.tensor([1.0, 2.0, 3.0], dtype=torch.float64, device=dev)
    with pytest.raises(B.SvdsError) as e:
        B.svds_create(rp, ci, va, 2, 2, on_device=True)
    assert e.value.code == B.SVDS_ERR_CSR


# ---------------------------------------------------------------- JDQMR
@pytest.mark.parametrize("target", ["smallest", "largest"])
def test_jdqmr_stage1_grid2d_closed_form(target):
    A = wl.grid_difference(32, 2)
    s = _grid_sigma(32, 2)
    ex = s[:5] if target == "smallest" else s[::-1][:5]
    r = B.svds(A, 5, target, 1e-10, maxBlockSize=2, method_stage1=B.SVDS_JDQMR, method_stage2=B.SVDS_JDQMR,
               initV=wl.start_block(A.n, 2, 0), maxMatvecs=400000)
    np.testing.assert_allclose(r["sigma"], ex, rtol=1e-10)
    _check_certificate(A, r, 1e-10, s[-1], 5)
    check_grid_vectors(A, 32, 2, r)
    assert r["stats"]["inner_steps"] > 0


@pytest.mark.parametrize("target", ["smallest", "largest"])
def test_jdqmr_stage2_tight_tolerance(target):
    A = wl.random_illconditioned(900, 300, 16, seed=13)
    r = B.svds(A, 3, target, 1e-13, maxBlockSize=2, method_stage1=B.SVDS_JDQMR, method_stage2=B.SVDS_JDQMR,
               initV=wl.start_block(A.n, 2, 2), maxMatvecs=600000)
    _compare_to_dense(A, r, target, 3, 1e-13)


def test_jdqmr_mixed_precision_3d_block4():
    A = wl.grid_difference(12, 3)
    s = _grid_sigma(12, 3)
    r = B.svds(A, 6, "smallest", 1e-10, maxBlockSize=4, method_stage1=B.SVDS_JDQMR, stage1_precision=B.SVDS_FP32,
               maxMatvecs=800000)
    np.testing.assert_allclose(r["sigma"], s[:6], rtol=1e-10)
    _check_certificate(A, r, 1e-10, s[-1], 6)
    check_grid_vectors(A, 12, 3, r)


def test_jdqmr_weighted_grid_jacobi():
    A = wl.weighted_grid(20, 2, seed=10001)
    sv = np.linalg.svd(A.to_scipy().toarray(), compute_uv=False)
    r = B.svds(A, 4, "smallest", 1e-10, maxBlockSize=2, method_stage1=B.SVDS_JDQMR, maxMatvecs=800000)
    np.testing.assert_allclose(r["sigma"], sv[::-1][:4], rtol=1e-10)
    _check_certificate(A, r, 1e-10, sv[0], 4)
    check_dense_vectors(A, r)


@pytest.mark.parametrize("target", ["smallest", "largest"])
def test_jdqmr_fp64_inner_solves(target):
    A = wl.random_illconditioned(1500, 500, 16, seed=11)
    r = B.svds(A, 4, target, 1e-10, maxBlockSize=4, method_stage1=B.SVDS_JDQMR, method_stage2=B.SVDS_JDQMR,
               innerPrecision=B.SVDS_DF64, maxMatvecs=600000)
    _compare_to_dense(A, r, target, 4, 1e-10)


@pytest.mark.parametrize("form", [dict(), dict(stage1_precision=B.SVDS_FP32, method_stage1=B.SVDS_JDQMR),
                                  dict(stage1_precision=B.SVDS_NATIVE_FP64)])
def test_explicit_normal_matrix_matches_two_passes(form):
    """C = A^T A as one explicit sparse matrix: same triplets as A then A^T."""
    A = wl.weighted_grid(20, 2, seed=5)
    out = {}
    for name, mode in (("two", B.SVDS_NORMAL_TWOPASS), ("explicit", B.SVDS_NORMAL_EXPLICIT)):
        r = B.svds(A, 5, "smallest", tol=1e-10, maxBlockSize=2, normalOperator=mode, **form)
        assert r["nconv"] == 5
        out[name] = r
    assert out["two"]["stats"]["normal_nnz"] == 0
    S = A.to_scipy()
    C = (S.T @ S).tocsr()
    assert out["explicit"]["stats"]["normal_nnz"] == C.nnz
    sd = np.sort(np.linalg.svd(S.toarray(), compute_uv=False))[:5]
    normA = np.linalg.norm(S.toarray(), 2)
    for name in ("two", "explicit"):
        np.testing.assert_allclose(out[name]["sigma"], sd, rtol=1e-10)
        _check_certificate(A, out[name], 1e-10, normA, 5)
        check_dense_vectors(A, out[name])


def test_auto_normal_operator_choice():
    """AUTO: explicit C for grid operators (few nonzeros per row of C), two passes
    for a matrix whose C is much denser than A."""
    g = wl.grid_difference(16, 3)
    r = B.svds(g, 3, "smallest", tol=1e-8, maxBlockSize=2)
    assert r["stats"]["normal_nnz"] > 0
    d = wl.random_illconditioned(3000, 1500, per_col=16, seed=3)
    r = B.svds(d, 3, "largest", tol=1e-8, maxBlockSize=2)
    assert r["stats"]["normal_nnz"] == 0


@pytest.mark.parametrize("target", ["smallest", "largest"])
def test_bf16_stage1_values_give_the_same_triplets(target):
    """Stage-1 operator with bfloat16 values (FP32 vectors), FP32 values and the
    FP64-class path: every form returns the same triplets to the tolerance;
    the per-triplet relative difference against the FP64-class form is checked."""
    A = wl.random_illconditioned(1500, 500, 16, seed=21)
    k = 4
    out = {}
    for name, prec in (("bf16", B.SVDS_BF16), ("fp32", B.SVDS_FP32), ("fp64", B.SVDS_DF64)):
        r = B.svds(A, k, target, 1e-10, maxBlockSize=2, stage1_precision=prec, method_stage1=B.SVDS_JDQMR,
                   initV=wl.start_block(A.n, 2, 3), maxMatvecs=600000)
        assert r["nconv"] == k, name
        _compare_to_dense(A, r, target, k, 1e-10)
        out[name] = r
    for name in ("bf16", "fp32"):
        # each form is within 1e-10 of the dense values, so within 2e-10 of each other
        rel = np.abs(out[name]["sigma"] - out["fp64"]["sigma"]) / out["fp64"]["sigma"]
        assert rel.max() <= 2e-10, (name, rel)


def test_bf16_exact_values_on_a_grid():
    """Grid operators have values +-1: bfloat16 is exact, the FP32 floor applies."""
    A = wl.grid_difference(24, 2)
    r = B.svds(A, 5, "smallest", 1e-10, maxBlockSize=2, stage1_precision=B.SVDS_BF16)
    s = np.sort(np.linalg.svd(A.to_scipy().toarray(), compute_uv=False))[:5]
    np.testing.assert_allclose(r["sigma"], s, rtol=1e-10)
    _check_certificate(A, r, 1e-10, _grid_sigma(24, 2)[-1], 5)
    check_grid_vectors(A, 24, 2, r)


@pytest.mark.parametrize("method", [B.SVDS_GDPK, B.SVDS_JDQMR])
def test_many_triplets(method):
    """A larger k (basis sizes grow with k + b): the 40 smallest triplets of a 2D
    grid against the closed form."""
    A = wl.grid_difference(24, 2)
    s = _grid_sigma(24, 2)
    r = B.svds(A, 40, "smallest", 1e-10, maxBlockSize=4, method_stage1=method, stage1_precision=B.SVDS_FP32,
               maxMatvecs=2000000)
    assert r["nconv"] == 40
    np.testing.assert_allclose(r["sigma"], s[:40], rtol=1e-10)
    _check_certificate(A, r, 1e-10, s[-1], 40)
    check_grid_vectors(A, 24, 2, r)


@pytest.mark.parametrize("target", ["smallest", "largest"])
def test_many_triplets_120(target):
    """The many-triplet regime (k = 120, basis 132 columns: tiled kernels beyond
    the 64-column row kernels) against the closed form of a 2D grid."""
    A = wl.grid_difference(40, 2)
    s = _grid_sigma(40, 2)
    ref = s[:120] if target == "smallest" else s[::-1][:120]
    r = B.svds(A, 120, target, 1e-10, maxBlockSize=4, method_stage1=B.SVDS_JDQMR, stage1_precision=B.SVDS_FP32,
               maxMatvecs=5000000)
    assert r["nconv"] == 120
    np.testing.assert_allclose(r["sigma"], ref, rtol=1e-10)
    _check_certificate(A, r, 1e-10, s[-1], 120)
    check_grid_vectors(A, 40, 2, r)


def _wide(A):
    At = A.to_scipy().T.tocsr()
    At.sort_indices()
    return wl.CSR(At.shape[0], At.shape[1], At.indptr.astype(np.int32), At.indices.astype(np.int32), At.data, "wide")


def _dense_kappa(A):
    s = np.linalg.svd(A.to_scipy().toarray(), compute_uv=False)
    return s[0], s[-1]


@pytest.mark.parametrize("prec", [B.SVDS_DF64, B.SVDS_FP32])
@pytest.mark.parametrize("method", [B.SVDS_GDPK, B.SVDS_JDQMR])
@pytest.mark.parametrize("name", ["grid3d", "random", "wide"])
def test_condest_within_the_relative_bound(prec, method, name):
    """svds_condest (Sec. 5, rel_tol 0.1).  Always: Ritz values lie inside the
    spectrum, so sigma_max is not overestimated, sigma_min not underestimated
    and the estimate never exceeds kappa.  Where the extreme values are well
    separated (3D grid, the wide random matrix) the relative rule at both ends
    puts it in [kappa sqrt(0.9 / 1.1), kappa], as the oracle's estimate on the
    same matrix; on the square random matrix, whose smallest values are
    clustered, a block-1 low-accuracy solve may stop at an interior value (the
    paper's caveat), so only the bounds are asserted.  With a tiny rel_tol the
    estimate is kappa to 1e-8.  The relative mode runs GD+k corrections for
    either stage-1 method (block-1 JDQMR with a loose stop can settle on an
    interior value)."""
    A = {"grid3d": lambda: wl.grid_difference(14, 3),
         "random": lambda: wl.random_illconditioned(3001, 1203, 16, seed=3),
         "wide": lambda: _wide(wl.random_illconditioned(1500, 600, 16, seed=5))}[name]()
    smax, smin = _dense_kappa(A)
    kappa = smax / smin
    r = B.condest(A, 0.1, stage1_precision=prec, method_stage1=method)
    assert r["rc"] == 0
    assert r["sigma_max"] <= smax * (1 + 1e-12) and r["sigma_min"] >= smin * (1 - 1e-12)
    assert r["kappa"] <= kappa * (1 + 1e-12)
    assert r["stats_largest"]["stage2_used"] == 0 and r["stats_smallest"]["stage2_used"] == 0
    if name != "random":
        assert kappa * np.sqrt(0.9 / 1.1) <= r["kappa"], (r["kappa"], kappa)
        o = O.condest(A.to_scipy(), 0.1)
        assert kappa * np.sqrt(0.9 / 1.1) <= o["kappa"] <= kappa * (1 + 1e-12)
    tight = B.condest(A, 1e-9, stage1_precision=prec, method_stage1=method)
    assert abs(tight["kappa"] / kappa - 1) < 1e-8, (tight["kappa"], kappa)


def test_relative_mode_counts_the_relative_rule():
    """svds_solve with relTol: the returned pairs meet ||C v - sigma^2 v|| <=
    relTol sigma^2 (checked in FP64 on the host), numConverged counts them."""
    A = wl.grid_difference(16, 3)
    for target in ("largest", "smallest"):
        r = B.svds(A, 3, target, 1e-10, maxBlockSize=1, relTol=0.05)
        S = A.to_scipy()
        V = r["V"]
        CV = S.T @ (S @ V)
        lam = np.sum(V * CV, axis=0)
        res = np.linalg.norm(CV - V * lam, axis=0)
        assert r["nconv"] == 3
        assert np.all(res <= 0.05 * lam * (1 + 1e-9) + 1e-12), (res, lam)
        np.testing.assert_allclose(r["sigma"] ** 2, lam, rtol=1e-12)


@pytest.mark.parametrize("target", ["smallest", "largest"])
def test_dynamic_method_closed_form(target):
    """DYNAMIC stage 1 (Sec. 3.4): the same triplets as the fixed methods (closed
    form of a 3D grid), and the switching uses both corrections."""
    A = wl.grid_difference(24, 3)
    s = _grid_sigma(24, 3)
    ref = s[:10] if target == "smallest" else s[::-1][:10]
    r = B.svds(A, 10, target, 1e-10, maxBlockSize=4, method_stage1=B.SVDS_DYNAMIC, stage1_precision=B.SVDS_FP32,
               maxMatvecs=5000000)
    assert r["nconv"] == 10
    np.testing.assert_allclose(r["sigma"], ref, rtol=1e-10)
    _check_certificate(A, r, 1e-10, s[-1], 10)
    check_grid_vectors(A, 24, 3, r)
    st = r["stats"]
    assert 0 < st["outer_stage1_jdqmr"] < st["outer_stage1"], st


def test_dynamic_method_mixes_the_two_corrections():
    """On a 64^3 grid (smallest, Jacobi) JDQMR needs few outer iterations and
    many products, GD+k the opposite.  DYNAMIC chooses per outer iteration, so
    it uses both corrections and lands between the fixed methods in both
    counts: fewer outer iterations than GD+k and fewer products than JDQMR."""
    A = wl.grid_difference(64, 3)
    s = _grid_sigma(64, 3)
    kw = dict(maxBlockSize=4, stage1_precision=B.SVDS_FP32, maxMatvecs=20000000)
    st = {}
    for name, m in (("gdk", B.SVDS_GDPK), ("jdqmr", B.SVDS_JDQMR), ("dynamic", B.SVDS_DYNAMIC)):
        r = B.svds(A, 10, "smallest", 1e-10, method_stage1=m, **kw)
        assert r["nconv"] == 10
        np.testing.assert_allclose(r["sigma"], s[:10], rtol=1e-10)
        st[name] = r["stats"]
    d = st["dynamic"]
    assert 0 < d["outer_stage1_jdqmr"] < d["outer_stage1"], d
    assert d["outer_stage1"] < st["gdk"]["outer_stage1"], st
    assert d["matvecs_stage1"] < st["jdqmr"]["matvecs_stage1"], st


@pytest.mark.parametrize("method", [B.SVDS_GDPK, B.SVDS_JDQMR])
@pytest.mark.parametrize("prec", [B.SVDS_DF64, B.SVDS_FP32])
def test_block_jacobi_preconditioner(method, prec):
    """Block Jacobi on A^T A (Sec. 4) in both stage-1 methods and precisions:
    the closed-form triplets of a 3D grid; with GD+k (one preconditioner
    application per product) fewer products than Jacobi.  JDQMR's fixed inner
    budget turns a better preconditioner into fewer products only sometimes,
    so there the count is not asserted."""
    A = wl.grid_difference(20, 3)
    s = _grid_sigma(20, 3)
    out = {}
    for pc in (B.SVDS_PRECOND_JACOBI, B.SVDS_PRECOND_BLOCKJACOBI):
        r = B.svds(A, 6, "smallest", 1e-10, maxBlockSize=2, method_stage1=method, stage1_precision=prec,
                   precond=pc, precondBlockSize=20, maxMatvecs=5000000)
        assert r["nconv"] == 6
        np.testing.assert_allclose(r["sigma"], s[:6], rtol=1e-10)
        _check_certificate(A, r, 1e-10, s[-1], 6)
        check_grid_vectors(A, 20, 3, r)
        out[pc] = r["stats"]["matvecs_stage1"]
    # blocks of 20 are whole grid lines: a stronger preconditioner than Jacobi
    if method == B.SVDS_GDPK:
        assert out[B.SVDS_PRECOND_BLOCKJACOBI] < out[B.SVDS_PRECOND_JACOBI], out
