"""Per-kernel parity of the CUDA path against the oracle / FP64 definitions.

Tolerances: FP64-class modes (DF64, F64) must agree normwise to 1e-13 relative
to ||(|A| |X|)|| (the FP64 SpMM accuracy bar of 1e-13, read normwise because
element-wise relative error is unbounded under cancellation); the F32 mode to a few units
of 2^-24 times the same normaliser.
"""
import numpy as np
import pytest

import oracle
from paper_1607_01404_gb300 import binding as B
from paper_1607_01404_gb300 import build as BLD
from paper_1607_01404_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from gpu_util import coef_device, csr_device, to_device, to_host  # noqa: E402

TOL = {B.PREC_F32: 2e-6, B.PREC_DF64: 1e-13, B.PREC_F64: 1e-13}
PRECS = [B.PREC_F32, B.PREC_DF64, B.PREC_F64]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    BLD.build()
    B.lib()


def _matrices():
    return [
        wl.random_illconditioned(3001, 1203, 16, seed=3),  # ragged rows, empty rows
        wl.grid_difference(9, 3),
        wl.weighted_grid(23, 2, seed=1),
    ]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("b", [1, 2, 3, 4, 5, 8, 11])
def test_spmm_matches_oracle(prec, b):
    for A in _matrices():
        d = csr_device(A)
        X = wl.dense_block(A.n, b, seed=b)
        Xd = to_device(prec, X)
        Xs = to_host(prec, Xd, A.n, b)  # the stored (rounded) input
        Yd = to_device(prec, np.zeros((A.m, b)))
        lo = None if d["exact"] else d["v32lo"]
        B.spmm(prec, A.m, A.n, d["rp"], d["ci"], d["v32"], lo, d["v64"], Xd, b, Yd, b, b)
        Y = to_host(prec, Yd, A.m, b)
        Aabs = A.to_scipy().copy()
        Aabs.data = np.abs(Aabs.data)
        norm = np.abs(Aabs @ np.abs(Xs)).max()
        ref = oracle.spmm(A, Xs)
        err = np.abs(Y - ref).max() / norm
        assert err <= TOL[prec], (A.name, err)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("b,col", [(4, 1), (4, 3), (8, 2), (2, 1)])
def test_spmm_into_unaligned_columns(prec, b, col):
    """Y = A X written into columns col .. col + b of a wider block (its rows do
    not start on 16-byte boundaries) from an aligned X: 16-byte gathers with
    element stores; the columns around the window keep their values."""
    for A in (wl.random_illconditioned(3001, 1203, 16, seed=3), wl.grid_difference(9, 3)):  # long and 2-entry rows
        _spmm_window(prec, A, b, col)


def _spmm_window(prec, A, b, col):
    d = csr_device(A)
    X = wl.dense_block(A.n, b, seed=b)
    Xd = to_device(prec, X)
    Xs = to_host(prec, Xd, A.n, b)
    ld = ((b + col + 3) // 4) * 4
    Y0 = wl.dense_block(A.m, ld, seed=7)
    Yd = to_device(prec, Y0)
    Yb = to_host(prec, Yd, A.m, ld)
    esz = 1 if prec == B.PREC_F32 or prec == B.PREC_F64 else 2
    lo = None if d["exact"] else d["v32lo"]
    B.spmm(prec, A.m, A.n, d["rp"], d["ci"], d["v32"], lo, d["v64"], Xd, b, Yd[col * esz:], ld, b)
    Y = to_host(prec, Yd, A.m, ld)
    Aabs = A.to_scipy().copy()
    Aabs.data = np.abs(Aabs.data)
    norm = np.abs(Aabs @ np.abs(Xs)).max()
    assert np.abs(Y[:, col:col + b] - oracle.spmm(A, Xs)).max() / norm <= TOL[prec]
    assert np.array_equal(Y[:, :col], Yb[:, :col]) and np.array_equal(Y[:, col + b:], Yb[:, col + b:])


@pytest.mark.parametrize("prec", [B.PREC_DF64, B.PREC_F64])
def test_spmm_transpose_and_ld(prec):
    A = wl.random_illconditioned(2000, 700, 16, seed=9)
    d = csr_device(A)
    # explicit transpose on the device, then A^T Y with strided blocks (ld > b)
    At = A.to_scipy().T.tocsr()
    At.sort_indices()
    AT = wl.CSR(A.n, A.m, At.indptr.astype(np.int32), At.indices.astype(np.int32), At.data, "AT")
    dt = csr_device(AT)
    b, ld = 4, 7
    Yh = wl.dense_block(A.m, ld, seed=5)
    Yd = to_device(prec, Yh)
    Ys = to_host(prec, Yd, A.m, ld)[:, :b]
    Xd = to_device(prec, np.zeros((A.n, ld)))
    B.spmm(prec, A.n, A.m, dt["rp"], dt["ci"], dt["v32"], None if dt["exact"] else dt["v32lo"], dt["v64"],
           Yd, ld, Xd, ld, b)
    X = to_host(prec, Xd, A.n, ld)
    ref = oracle.spmm_t(A, Ys)
    Aabs = abs(At)
    norm = np.abs(Aabs @ np.abs(Ys)).max()
    assert np.abs(X[:, :b] - ref).max() / norm <= TOL[prec]
    assert np.all(X[:, b:] == 0)  # columns beyond b untouched


def test_csr_transpose_bit_exact_and_deterministic():
    for A in _matrices() + [wl.random_illconditioned(500, 20, 16, seed=1)]:  # long columns use heapsort path
        d = csr_device(A)
        dev = d["rp"].device
        rpT = torch.zeros(A.n + 1, dtype=torch.int32, device=dev)
        ciT = torch.zeros(max(A.nnz, 1), dtype=torch.int32, device=dev)
        vaT = torch.zeros(max(A.nnz, 1), dtype=torch.float64, device=dev)
        work = torch.zeros(B.csr_transpose_work_bytes(A.n), dtype=torch.uint8, device=dev)
        B.csr_transpose(A.m, A.n, d["rp"], d["ci"], d["va"], rpT, ciT, vaT, work)
        torch.cuda.synchronize()
        S = A.to_scipy()
        # definition: entry (i, j) of A becomes (j, i); rows of A^T sorted by i
        rows = np.repeat(np.arange(A.m), np.diff(A.rowptr))
        order = np.lexsort((rows, A.colidx))
        ref_ci = rows[order]
        ref_va = A.vals[order]
        ref_rp = np.concatenate([[0], np.cumsum(np.bincount(A.colidx, minlength=A.n))])
        assert np.array_equal(rpT.cpu().numpy(), ref_rp)
        assert np.array_equal(ciT.cpu().numpy()[:A.nnz], ref_ci)
        assert np.array_equal(vaT.cpu().numpy()[:A.nnz], ref_va)
        ci1 = ciT.clone()
        B.csr_transpose(A.m, A.n, d["rp"], d["ci"], d["va"], rpT, ciT, vaT, work)
        torch.cuda.synchronize()
        assert torch.equal(ci1, ciT)
        assert S.shape == (A.m, A.n)


def _ld(p, aligned):
    """Leading dimension: a multiple of 4 elements takes the tiled (cp.async) path,
    p + 3 (odd row stride) the generic path."""
    return ((p + 3) // 4) * 4 if aligned else p + 3


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("aligned", [True, False])
@pytest.mark.parametrize("p,q,r0,r1", [(35, 4, 0, 100003), (9, 1, 17, 5000), (3, 8, 0, 1), (40, 13, 5, 77777),
                                       (256, 2, 0, 3000), (7, 3, 64, 64), (32, 4, 0, 70001), (64, 7, 3, 50000)])
@pytest.mark.parametrize("pshift,qshift", [(0, 0), (0, 1), (1, 1)])
def test_gram_matches_fp64(prec, aligned, p, q, r0, r1, pshift, qshift):
    L = max(r1, 10)
    P = wl.dense_block(L, p + pshift, seed=1)
    Q = wl.dense_block(L, q + qshift, seed=2)
    ldp, ldq = _ld(p + pshift, aligned), _ld(q + qshift, aligned)
    Pd, Qd = to_device(prec, P, ld=ldp), to_device(prec, Q, ld=ldq)
    Ps = to_host(prec, Pd, L, ldp)[:, pshift:p + pshift]
    Qs = to_host(prec, Qd, L, ldq)[:, qshift:q + qshift]
    G = torch.zeros(p * q, dtype=torch.float64, device="cuda:0")
    scratch = torch.zeros(B.gram_scratch_bytes(p, q), dtype=torch.uint8, device="cuda:0")
    esz = 1 if prec == B.PREC_F32 or prec == B.PREC_F64 else 2
    # P and Q start at columns pshift and qshift: 1 is a window that is not
    # 16-byte aligned inside its rows
    B.gram(prec, r0, r1, Pd[pshift * esz:], ldp, p, Qd[qshift * esz:], ldq, q, G, scratch)
    Gh = G.cpu().numpy().reshape(p, q)
    ref = Ps[r0:r1].T @ Qs[r0:r1]
    norm = np.abs(Ps[r0:r1]).T @ np.abs(Qs[r0:r1])
    # FP64-class accumulation in every mode
    assert np.all(np.abs(Gh - ref) <= 1e-13 * norm + 1e-300)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("aligned", [True, False])
@pytest.mark.parametrize("p,q", [(21, 4), (35, 1), (6, 8), (44, 30)])
def test_combine_and_inplace_restart(prec, aligned, p, q):
    L = 20011
    ldp, ldq = _ld(p, aligned), _ld(q, aligned)
    P = wl.dense_block(L, p, seed=3)
    In = wl.dense_block(L, q, seed=4)
    Cm = wl.dense_block(p, q, seed=5)
    R = np.triu(wl.dense_block(q, q, seed=6)) + 3 * np.eye(q)
    Ri = np.linalg.inv(R)
    Pd, Ind = to_device(prec, P, ld=ldp), to_device(prec, In, ld=ldq)
    Ps, Ins = to_host(prec, Pd, L, ldp)[:, :p], to_host(prec, Ind, L, ldq)[:, :q]
    Cd, Rd = coef_device(prec, Cm), coef_device(prec, Ri)
    Out = to_device(prec, np.zeros((L, ldq)))
    B.combine(prec, L, Pd, ldp, p, Cd, Ind, ldq, 1, Out, ldq, q, Rd)
    got = to_host(prec, Out, L, ldq)[:, :q]
    ref = (Ins + Ps @ Cm) @ Ri
    scale = (np.abs(Ins) + np.abs(Ps) @ np.abs(Cm)) @ np.abs(Ri)
    assert np.all(np.abs(got - ref) <= 4 * TOL[prec] * scale)
    # without R^-1 and without In
    Out2 = to_device(prec, np.zeros((L, ldq)))
    B.combine(prec, L, Pd, ldp, p, Cd, None, 0, 0, Out2, ldq, q)
    got = to_host(prec, Out2, L, ldq)[:, :q]
    assert np.all(np.abs(got - Ps @ Cm) <= 4 * TOL[prec] * (np.abs(Ps) @ np.abs(Cm)))
    # in place: V <- V Z (columns <= p) writes the first columns of P's own buffer
    nz = min(p, 7)
    Z = np.linalg.qr(wl.dense_block(p, nz, seed=7))[0]
    Zd = coef_device(prec, Z)
    B.combine(prec, L, Pd, ldp, p, Zd, None, 0, 0, Pd, ldp, nz)
    got = to_host(prec, Pd, L, ldp)[:, :p]
    ref = Ps @ Z
    assert np.abs(got[:, :nz] - ref).max() <= 4 * TOL[prec] * (np.abs(Ps) @ np.abs(Z)).max()
    assert np.array_equal(got[:, nz:], Ps[:, nz:])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("L", [1, 255, 256, 257, 100003])
@pytest.mark.parametrize("p,q", [(1, 1), (4, 3), (32, 4), (32, 18), (35, 5), (64, 12), (64, 32), (17, 23)])
def test_combine_row_tiles(prec, L, p, q):
    """Out = In + P C on 16-byte-aligned blocks (the TMA-fed update: 256-row
    tiles, ragged last tile, every output-width bucket), then the in-place CGS
    step T <- (T - V C) R^-1 with Out = In, and the in-place restart V <- V Z."""
    ldp, ldq = ((p + 3) // 4) * 4, ((q + 3) // 4) * 4
    P = wl.dense_block(L, p, seed=13)
    T = wl.dense_block(L, q, seed=14)
    Cm = wl.dense_block(p, q, seed=15)
    Pd, Td = to_device(prec, P, ld=ldp), to_device(prec, T, ld=ldq)
    Ps, Ts = to_host(prec, Pd, L, ldp)[:, :p], to_host(prec, Td, L, ldq)[:, :q]
    Cd = coef_device(prec, Cm)
    Out = to_device(prec, np.zeros((L, ldq)))
    B.combine(prec, L, Pd, ldp, p, Cd, Td, ldq, 1, Out, ldq, q)
    got = to_host(prec, Out, L, ldq)[:, :q]
    scale = np.abs(Ts) + np.abs(Ps) @ np.abs(Cm)
    assert np.all(np.abs(got - (Ts + Ps @ Cm)) <= 4 * TOL[prec] * scale)
    if q <= 8:
        R = np.triu(wl.dense_block(q, q, seed=16)) + 3 * np.eye(q)
        Ri = np.linalg.inv(R)
        B.combine(prec, L, Pd, ldp, p, coef_device(prec, -Cm), Td, ldq, 1, Td, ldq, q, coef_device(prec, Ri))
        got = to_host(prec, Td, L, ldq)[:, :q]
        ref = (Ts - Ps @ Cm) @ Ri
        sc = (np.abs(Ts) + np.abs(Ps) @ np.abs(Cm)) @ np.abs(Ri)
        assert np.all(np.abs(got - ref) <= 4 * TOL[prec] * sc)
    nz = min(p, q)
    Z = np.linalg.qr(wl.dense_block(p, p, seed=17))[0][:, :nz]
    B.combine(prec, L, Pd, ldp, p, coef_device(prec, Z), None, 0, 0, Pd, ldp, nz)
    got = to_host(prec, Pd, L, ldp)[:, :p]
    assert np.all(np.abs(got[:, :nz] - Ps @ Z) <= 4 * TOL[prec] * (np.abs(Ps) @ np.abs(Z)))
    assert np.array_equal(got[:, nz:], Ps[:, nz:])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("aligned", [True, False])
@pytest.mark.parametrize("g,nb", [(35, 4), (6, 1), (17, 3), (44, 8), (20, 13), (32, 4), (64, 8), (1, 2), (64, 5)])
def test_ritz_residual(prec, aligned, g, nb):
    L = 50001
    ldv = _ld(g, aligned)
    V = wl.dense_block(L, g, seed=8)
    W = wl.dense_block(L, g, seed=9)
    Y = wl.dense_block(g, nb, seed=10)
    th = wl.dense_block(nb, 1, seed=11).ravel()
    Vd, Wd = to_device(prec, V, ld=ldv), to_device(prec, W, ld=ldv)
    Vs, Ws = to_host(prec, Vd, L, ldv)[:, :g], to_host(prec, Wd, L, ldv)[:, :g]
    Yd, Td = coef_device(prec, Y), coef_device(prec, th)
    Xd, Rd = to_device(prec, np.zeros((L, nb))), to_device(prec, np.zeros((L, nb)))
    n2 = torch.zeros(nb, dtype=torch.float64, device="cuda:0")
    scratch = torch.zeros(B.ritz_scratch_bytes(nb), dtype=torch.uint8, device="cuda:0")
    B.ritz_residual(prec, L, Vd, Wd, ldv, g, Yd, Td, Xd, Rd, nb, nb, n2, scratch)
    X, R = to_host(prec, Xd, L, nb), to_host(prec, Rd, L, nb)
    Xr = Vs @ Y
    Rr = Ws @ Y - Xr * th
    sx = np.abs(Vs) @ np.abs(Y)
    assert np.all(np.abs(X - Xr) <= 4 * TOL[prec] * sx)
    assert np.all(np.abs(R - Rr) <= 4 * TOL[prec] * (np.abs(Ws) @ np.abs(Y) + sx * np.abs(th)))
    nr = np.sum(R * R, axis=0)
    np.testing.assert_allclose(n2.cpu().numpy(), nr, rtol=1e-12)


@pytest.mark.parametrize("b", [1, 2, 4, 8, 5])
def test_spmm_bf16_values_match_oracle(b):
    """bfloat16 values: bit-exact rounding against the oracle's definition, and
    Y = bf16(A) X in FP32 against the FP64 product with the rounded values."""
    from oracle.phsvds_fp64 import round_bf16

    for A in _matrices():
        d = csr_device(A)
        v16 = torch.zeros(max(A.nnz, 1), dtype=torch.int16, device=d["v32"].device)
        flags = torch.zeros(4, dtype=torch.int32, device=d["v32"].device)
        B.to_bf16(d["v32"][: A.nnz], v16, flags)
        torch.cuda.synchronize()
        v32 = A.vals.astype(np.float32)
        r16 = round_bf16(v32)
        got = (v16[: A.nnz].cpu().numpy().astype(np.uint16).astype(np.uint32) << 16).view(np.float32)
        np.testing.assert_array_equal(got, r16)
        assert int(flags[0].item()) == int(np.any(r16 != v32))
        X = wl.dense_block(A.n, b, seed=b).astype(np.float32).astype(np.float64)
        Xd = torch.from_numpy(X.astype(np.float32).ravel()).to(d["v32"].device)
        Yd = torch.zeros(A.m * b, dtype=torch.float32, device=d["v32"].device)
        B.spmm_bf16(A.m, A.n, d["rp"], d["ci"], v16, Xd, b, Yd, b, b)
        Y = Yd.cpu().numpy().astype(np.float64).reshape(A.m, b)
        Ar = wl.CSR(A.m, A.n, A.rowptr, A.colidx, r16.astype(np.float64), A.name)
        ref = oracle.spmm(Ar, X)
        Aabs = Ar.to_scipy().copy()
        Aabs.data = np.abs(Aabs.data)
        norm = np.abs(Aabs @ np.abs(X)).max()
        assert np.abs(Y - ref).max() / norm <= TOL[B.PREC_F32], A.name


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("g,nb", [(7, 4), (33, 4), (20, 1), (12, 8)])
def test_device_ortho_matches_oracle(prec, g, nb):
    """Device CGS2 + CholQR2 of a block against an orthonormal basis: the unique
    Q of T = V C + Q R (R with positive diagonal), as the oracle computes it."""
    L = 30011
    rng = np.random.default_rng(g * 10 + nb)
    V = np.linalg.qr(rng.standard_normal((L, g)))[0]
    T = rng.standard_normal((L, nb)) + V @ rng.standard_normal((g, nb))  # with components along V
    ldv, ldt = _ld(g, True), _ld(nb, True)
    Vd, Td = to_device(prec, V, ld=ldv), to_device(prec, T, ld=ldt)
    Vs, Ts = to_host(prec, Vd, L, ldv)[:, :g], to_host(prec, Td, L, ldt)[:, :nb]
    status = B.ortho(prec, L, Vd, ldv, g, Td, ldt, nb)
    Q = to_host(prec, Td, L, ldt)[:, :nb]
    ref = oracle.orthonormalize(Ts, Vs)
    tol = 2e-5 if prec == B.PREC_F32 else 1e-11
    assert status == 0
    assert np.abs(Q - ref).max() <= tol, np.abs(Q - ref).max()
    assert np.abs(Q.T @ Q - np.eye(nb)).max() <= tol
    assert np.abs(Vs.T @ Q).max() <= tol


@pytest.mark.parametrize("prec", PRECS)
def test_device_ortho_breakdown_is_reported_and_repaired(prec):
    """A block with a column in span(V) and a duplicated column: the device
    CGS2 + CholQR2 reports the breakdown (host-visible status), and the
    solver's repair replaces the dependent columns by seeded random vectors
    so that the result is orthonormal and orthogonal to V; the independent
    column keeps its direction (it is the first column of Q up to sign)."""
    L, g, nb = 20011, 9, 4
    rng = np.random.default_rng(77)
    V = np.linalg.qr(rng.standard_normal((L, g)))[0]
    t = rng.standard_normal(L)
    T = np.stack([t, V @ rng.standard_normal(g), t, rng.standard_normal(L)], axis=1)  # col 1 in span(V), col 2 = col 0
    ldv, ldt = _ld(g, True), _ld(nb, True)
    Vd = to_device(prec, V, ld=ldv)
    Vs = to_host(prec, Vd, L, ldv)[:, :g]
    Td = to_device(prec, T, ld=ldt)
    assert B.ortho(prec, L, Vd, ldv, g, Td, ldt, nb) != 0
    Td = to_device(prec, T, ld=ldt)
    Ts = to_host(prec, Td, L, ldt)[:, :nb]
    status, replaced = B.ortho_repair(prec, L, Vd, ldv, g, Td, ldt, nb, seed=5)
    assert status != 0 and replaced == 1
    Q = to_host(prec, Td, L, ldt)[:, :nb]
    tol = 2e-5 if prec == B.PREC_F32 else 1e-11
    assert np.abs(Q.T @ Q - np.eye(nb)).max() <= tol
    assert np.abs(Vs.T @ Q).max() <= tol
    t0 = Ts[:, 0] - Vs @ (Vs.T @ Ts[:, 0])
    assert abs(abs(Q[:, 0] @ t0) / np.linalg.norm(t0) - 1) <= tol
    # a regular block goes through unchanged by the repair path
    Tr = rng.standard_normal((L, nb))
    Td = to_device(prec, Tr, ld=ldt)
    assert B.ortho_repair(prec, L, Vd, ldv, g, Td, ldt, nb) == (0, 0)


@pytest.mark.parametrize("bs", [1, 7, 32, 64])
@pytest.mark.parametrize("name", ["random", "grid"])
def test_block_jacobi_matches_oracle(bs, name):
    """CSR of the block-Jacobi inverse of A^T A (ragged last block, an empty
    column in the random matrix) against the oracle's dense block inverses."""
    import scipy.sparse as sp

    from oracle import phsvds_fp64 as O

    if name == "random":
        S = wl.random_illconditioned(2000, 701, 8, seed=bs).to_scipy().tolil()
        S[:, 300] = 0.0
        S = S.tocsr()
    else:
        S = wl.grid_difference(9, 3).to_scipy()
    S.eliminate_zeros()
    n = S.shape[1]
    At = S.T.tocsr()
    At.sort_indices()
    dev = torch.device("cuda:0")
    rpT = torch.from_numpy(At.indptr.astype(np.int32)).to(dev)
    ciT = torch.from_numpy(At.indices.astype(np.int32)).to(dev)
    vT = torch.from_numpy(At.data.astype(np.float64)).to(dev)
    nz = B.block_jacobi_nnz(n, bs)
    rp = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    ci = torch.zeros(nz, dtype=torch.int32, device=dev)
    v64 = torch.zeros(nz, dtype=torch.float64, device=dev)
    v32 = torch.zeros(nz, dtype=torch.float32, device=dev)
    B.block_jacobi(n, rpT, ciT, vT, bs, rp, ci, v64=v64, v32=v32)
    torch.cuda.synchronize()
    M = sp.csr_matrix((v64.cpu().numpy(), ci.cpu().numpy(), rp.cpu().numpy()), shape=(n, n))
    ref = O.block_jacobi(S, bs)
    assert np.array_equal(M.indptr, ref.indptr) and np.array_equal(M.indices, ref.indices)
    # FP64 Gauss-Jordan vs LAPACK inverse of each block: relative to the block's
    # largest entry, scaled by the block's condition number
    D = (M - ref).toarray()
    R = ref.toarray()
    for g0 in range(0, n, bs):
        I = slice(g0, min(n, g0 + bs))
        blk = R[I, I]
        kappa = np.linalg.cond(blk)
        assert np.abs(D[I, I]).max() <= 1e-14 * kappa * np.abs(blk).max() + 1e-300, (g0, kappa)
    np.testing.assert_array_equal(v32.cpu().numpy(), v64.cpu().numpy().astype(np.float32))
