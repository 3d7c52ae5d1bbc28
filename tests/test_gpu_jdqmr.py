"""GPU parity of the JDQMR inner solve (block symmetric QMR on the projected
correction equation) against the exact solution of that equation (oracle)."""
import numpy as np
import pytest

from gpu_util import coef_device, csr_device, to_device, to_host, torch_dev
from oracle.phsvds_fp64 import jd_correction_exact
from paper_1607_01404_gb300 import binding as B
from paper_1607_01404_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# converged inner solves: relative error of t against the exact solution
TOL = {B.PREC_F32: 2e-3, B.PREC_DF64: 1e-8, B.PREC_F64: 1e-9}


def _problem(nb, seed):
    A = wl.random_illconditioned(700, 240, per_col=6, seed=seed, umin=-1.0)
    S = A.to_scipy()
    C = (S.T @ S).tocsr()
    C.sort_indices()
    n = C.shape[0]
    lam = np.linalg.eigvalsh(C.toarray())
    rng = np.random.default_rng(seed)
    X = np.linalg.qr(rng.standard_normal((n, nb)))[0]
    Bm = rng.standard_normal((n, nb))
    Bm -= X * np.sum(X * Bm, axis=0)
    # shifts: below the spectrum (C - eta I definite) for even columns, in the
    # middle of the widest gap of the spectrum (indefinite) for odd ones
    g = int(np.argmax(np.diff(lam)))
    eta = np.array([-0.3 * lam.mean() if j % 2 == 0 else 0.5 * (lam[g] + lam[g + 1]) for j in range(nb)])
    Cw = wl.CSR(n, n, C.indptr.astype(np.int32), C.indices.astype(np.int32), C.data, "C")
    return Cw, C, X, Bm, eta


@pytest.mark.parametrize("prec", [B.PREC_F32, B.PREC_DF64, B.PREC_F64])
@pytest.mark.parametrize("nb", [1, 3, 4])
@pytest.mark.parametrize("jacobi", [False, True])
def test_inner_solve_converges_to_the_exact_correction(prec, nb, jacobi):
    torch, dev = torch_dev()
    Cw, C, X, Bm, eta = _problem(nb, seed=7 + nb)
    n = Cw.m
    d = csr_device(Cw)
    Xd, Bd = to_device(prec, X), to_device(prec, Bm)
    Td = to_device(prec, np.zeros((n, nb)))
    dinv = to_device(prec, (1.0 / C.diagonal())[:, None]) if jacobi else None
    lo = None if d["exact"] else d["v32lo"]
    steps = B.jd_solve(prec, n, d["rp"], d["ci"], d["v32"], lo, d["v64"], nb, Xd, Bd, eta, dinv, 600, 1e-13, Td)
    T = to_host(prec, Td, n, nb)
    ref = jd_correction_exact(C, X, Bm, eta)
    for j in range(nb):
        err = np.linalg.norm(T[:, j] - ref[:, j]) / np.linalg.norm(ref[:, j])
        assert err <= TOL[prec], (prec, nb, jacobi, j, err, steps)
        otol = 1e-3 if prec == B.PREC_F32 else 1e-9
        assert abs(X[:, j] @ T[:, j]) <= otol * np.linalg.norm(T[:, j])


def test_inner_solve_stops_on_the_relative_tolerance():
    torch, dev = torch_dev()
    Cw, C, X, Bm, eta = _problem(4, seed=3)
    n = Cw.m
    d = csr_device(Cw)
    Xd, Bd = to_device(B.PREC_DF64, X), to_device(B.PREC_DF64, Bm)
    Td = to_device(B.PREC_DF64, np.zeros((n, 4)))
    lo = None if d["exact"] else d["v32lo"]
    s_loose = B.jd_solve(B.PREC_DF64, n, d["rp"], d["ci"], d["v32"], lo, d["v64"], 4, Xd, Bd, eta, None, 600, 0.1, Td)
    s_tight = B.jd_solve(B.PREC_DF64, n, d["rp"], d["ci"], d["v32"], lo, d["v64"], 4, Xd, Bd, eta, None, 600, 1e-10,
                         Td)
    assert 0 < s_loose < s_tight <= 600


@pytest.mark.parametrize("prec", [B.PREC_F32, B.PREC_DF64, B.PREC_F64])
@pytest.mark.parametrize("nb", [1, 2, 4, 8])
@pytest.mark.parametrize("wide", [False, True])
def test_fused_operator_and_dots_match_fp64(prec, nb, wide):
    """W = K X with the four dot products of one inner step, E1 = x, E2 = q:
    [x^T w, q^T w, x^T q, q^T q] per column, against FP64 on the stored inputs."""
    torch, dev = torch_dev()
    A = wl.weighted_grid(41, 2, seed=nb)  # n = 1681: several CTAs and a ragged last one
    S = A.to_scipy()
    C = (S.T @ S).tocsr()
    C.sort_indices()
    n = C.shape[0]
    K = wl.CSR(n, n, C.indptr.astype(np.int32), C.indices.astype(np.int32), C.data, "C")
    d = csr_device(K)
    rng = np.random.default_rng(nb + 10 * wide)
    ldx = 2 * nb if wide else nb
    Xd = to_device(prec, rng.standard_normal((n, ldx)))
    E1d = to_device(prec, rng.standard_normal((n, nb)))
    E2d = to_device(prec, rng.standard_normal((n, nb)))
    X = to_host(prec, Xd, n, ldx)[:, :nb]
    E1, E2 = to_host(prec, E1d, n, nb), to_host(prec, E2d, n, nb)
    Wd = to_device(prec, np.zeros((n, nb)))
    dots = torch.zeros(4 * nb, dtype=torch.float64, device=dev)
    scratch = torch.zeros(B.spmm_dots_scratch_bytes(nb), dtype=torch.uint8, device=dev)
    B.spmm_dots(prec, n, d["rp"], d["ci"], d["v32"], None if d["exact"] else d["v32lo"], d["v64"], nb, Xd, ldx,
                Wd, E1d, E2d, dots, scratch)
    W = to_host(prec, Wd, n, nb)
    ref = C @ X
    norm = np.abs(abs(C) @ np.abs(X)).max()
    tw = 2e-6 if prec == B.PREC_F32 else 1e-13
    assert np.abs(W - ref).max() <= tw * norm
    got = dots.cpu().numpy().reshape(4, nb)
    Ws = W  # the dots use the stored W
    want = np.array([np.sum(E1 * Ws, 0), np.sum(E2 * Ws, 0), np.sum(E1 * E2, 0), np.sum(E2 * E2, 0)])
    scale = np.array([np.sum(np.abs(E1 * Ws), 0), np.sum(np.abs(E2 * Ws), 0), np.sum(np.abs(E1 * E2), 0),
                      np.sum(E2 * E2, 0)])
    td = 2e-5 if prec == B.PREC_F32 else 1e-13
    assert np.all(np.abs(got - want) <= td * scale), np.abs(got - want) / scale
