"""FP64 CPU oracle of PHSVDS (test infrastructure, never on the product path).

Follows the paper section by section:

* operators ``C = A^T A`` and ``B = [0 A^T; A 0]`` (Sec. 2.1, Eq. 2.4-2.5);
* the triplet residual (Eq. res, Sec. 3.1) and the stage-1 / stage-2
  convergence criteria (Algorithm 1 lines 2 and 18, Eq. B_secondCriterion);
* GD+k with soft locking on C, followed by a Rayleigh-Ritz on the returned
  vectors (Algorithm 1 lines 1-8, Sec. 3.2);
* the reset of V and W when a residual falls below sqrt(restarts) ||op|| eps
  (Sec. 3.2);
* stage 2 on B from the initial guesses [v; u]/sqrt(2) (Algorithm 1 line 9),
  with Rayleigh-Ritz for the largest and the simplified refined extraction with
  constant shift, incremental QR of (B - tau I)V, QR restart via QR(RY) and
  hard locking with a forced restart for the smallest (Sec. 3.1-3.2,
  Algorithm 1 lines 10-20).

Orthogonalisation is classical Gram-Schmidt applied twice followed by
Cholesky-QR applied twice.  The small dense problems use numpy/scipy LAPACK
routines (eigh, svd, qr, cholesky) as library steps.

Readings where the paper is silent (norm estimate, stagnation floor constant,
preconditioners, basis sizes for large k, block refined extraction, reported
sigma) are the ones listed in the design notes of this repository and are
repeated at the function that uses them.

Parity status: the operators, orthonormalisation and residual are pinned by
closed forms and dense LAPACK SVDs in the CPU tests; the iteration counts are
parity unpinned (they affect only speed, never the returned triplets).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

# Machine precision of the paper's runs (Sec. 4: 2.2e-16).
EPS = float(np.finfo(np.float64).eps)
# Stagnation floor constant: the paper observes stagnation below 10 ||C|| eps
# after the V/W reset (Sec. 3.2); Algorithm 1 line 2 writes eps ||C||.
FLOOR_C = 10.0


def _as_csr(A) -> sp.csr_matrix:
    if sp.issparse(A):
        return sp.csr_matrix(A, dtype=np.float64)
    if hasattr(A, "to_scipy"):
        return A.to_scipy()
    return sp.csr_matrix(np.asarray(A, dtype=np.float64))


# ----------------------------------------------------------------------------
# Operators (Sec. 2.1)
# ----------------------------------------------------------------------------
def spmm(A, X):
    """Y = A X, y_i = sum_j a_ij x_j (the user matvec of Sec. 3.4, transpose = 0)."""
    return _as_csr(A) @ X


def round_bf16(x):
    """bfloat16 rounding of FP32 values: keep the upper 16 bits of the IEEE
    single encoding after rounding to nearest, ties to even (the storage format
    of the reduced-precision operator; not in the paper).  Returns float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32)


def jd_correction_exact(C, X, B, eta):
    """Exact solution of the Jacobi-Davidson correction equation per column j
    (Sec. 3.4, JDQMR's inner system):
        (I - x_j x_j^T)(C - eta_j I)(I - x_j x_j^T) t_j = b_j,  t_j orthogonal to x_j,
    for unit vectors x_j and b_j orthogonal to x_j: t_j = Q (Q^T (C - eta_j I) Q)^-1 Q^T b_j
    with Q an orthonormal basis of the complement of x_j (dense; small n only)."""
    Cd = C.toarray() if hasattr(C, "toarray") else np.asarray(C, dtype=np.float64)
    n = Cd.shape[0]
    T = np.zeros_like(B, dtype=np.float64)
    for j in range(B.shape[1]):
        x = X[:, j] / np.linalg.norm(X[:, j])
        Qf, _ = np.linalg.qr(np.column_stack([x, np.eye(n)]))
        Q = Qf[:, 1:n]
        Mj = Q.T @ (Cd - eta[j] * np.eye(n)) @ Q
        T[:, j] = Q @ np.linalg.solve(Mj, Q.T @ B[:, j])
    return T


def spmm_t(A, Y):
    """X = A^T Y (the user matvec of Sec. 3.4 with transpose != 0)."""
    return _as_csr(A).T @ Y


def apply_C(A, X):
    """Normal-equations operator C = A^T A (Sec. 2.1; Algorithm 1 line 1)."""
    A = _as_csr(A)
    return A.T @ (A @ X)


def apply_B(A, X):
    """Augmented operator B = [0 A^T; A 0] on X = [X_v; X_u] (Eq. 2.4-2.5).

    The first n rows hold the right-vector part, the last m the left part.
    """
    A = _as_csr(A)
    n = A.shape[1]
    return np.vstack([A.T @ X[n:], A @ X[:n]])


def triplet_residuals(A, sigma, U, V):
    """||r_i|| = sqrt(||A v_i - s_i u_i||^2 + ||A^T u_i - s_i v_i||^2) (Eq. res)."""
    A = _as_csr(A)
    r1 = A @ V - U * sigma
    r2 = A.T @ U - V * sigma
    return np.sqrt(np.sum(r1 * r1, axis=0) + np.sum(r2 * r2, axis=0))


# ----------------------------------------------------------------------------
# ||A|| estimate (the paper uses ||A||_2 in every tolerance but does not say how
# it is obtained; reading: Lanczos with full reorthogonalisation on C)
# ----------------------------------------------------------------------------
def estimate_norm(A, seed: int = 7, maxit: int = 50, rtol: float = 1e-8) -> float:
    A = _as_csr(A)
    n = A.shape[1]
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(n)
    q /= np.linalg.norm(q)
    Qs = [q]
    alphas, betas = [], []
    prev = 0.0
    theta = 0.0
    for j in range(min(maxit, n)):
        w = A.T @ (A @ Qs[-1])
        alphas.append(float(Qs[-1] @ w))
        Qm = np.array(Qs).T
        for _ in range(2):  # full reorthogonalisation
            w = w - Qm @ (Qm.T @ w)
        beta = float(np.linalg.norm(w))
        T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
        theta = float(np.linalg.eigvalsh(T)[-1])
        if j > 0 and abs(theta - prev) <= rtol * theta:
            break
        prev = theta
        if beta <= 1e-14 * math.sqrt(max(theta, 1e-300)):
            break
        betas.append(beta)
        Qs.append(w / beta)
    return math.sqrt(max(theta, 0.0))


# ----------------------------------------------------------------------------
# Orthonormalisation: CGS applied twice, then Cholesky-QR applied twice
# ----------------------------------------------------------------------------
def _cholqr(T):
    G = T.T @ T
    Lc = np.linalg.cholesky(G)  # G = L L^T, R = L^T
    return sla.solve_triangular(Lc, T.T, lower=True).T


def orthonormalize(T, V=None, rng=None, drop_tol: float = 1e-10):
    """Return an orthonormal basis of (I - V V^T) T, with V orthonormal.

    CGS2 against V, then CholQR2.  A column that keeps less than ``drop_tol`` of
    its norm after the projection is replaced by a random vector (projected as
    well); if Cholesky still fails, a Householder QR is used for that block.
    """
    if rng is None:
        rng = np.random.default_rng(12345)
    T = np.array(T, dtype=np.float64, copy=True)
    if T.ndim == 1:
        T = T[:, None]
    norms0 = np.linalg.norm(T, axis=0)

    def project(X):
        if V is not None and V.shape[1] > 0:
            for _ in range(2):
                X = X - V @ (V.T @ X)
        return X

    T = project(T)
    bad = np.linalg.norm(T, axis=0) <= drop_tol * np.maximum(norms0, 1e-300)
    if np.any(bad):
        T[:, bad] = project(rng.standard_normal((T.shape[0], int(bad.sum()))))
    try:
        for _ in range(2):
            T = _cholqr(T)
    except np.linalg.LinAlgError:
        Qh, Rh = np.linalg.qr(T)
        small = np.abs(np.diag(Rh)) <= drop_tol * max(np.abs(np.diag(Rh)).max(), 1e-300)
        if np.any(small):
            Qh[:, small] = project(rng.standard_normal((T.shape[0], int(small.sum()))))
            Qh = project(Qh)
            Qh, _ = np.linalg.qr(Qh)
        T = Qh
    return T


def _orth_coeff(Y):
    """Orthonormal basis of the columns of a small coefficient matrix (restart)."""
    Q, R = np.linalg.qr(Y)
    keep = np.abs(np.diag(R)) > 1e-12 * max(1.0, np.abs(np.diag(R)).max())
    return Q[:, keep]


# ----------------------------------------------------------------------------
# GD+k with Rayleigh-Ritz extraction and soft locking
# ----------------------------------------------------------------------------
@dataclass
class Stats:
    outer: int = 0
    matvecs: int = 0  # products with A or A^T, one per column (the paper's "MV")
    restarts: int = 0
    resets: int = 0
    extra: dict = field(default_factory=dict)


def _sort_order(theta, target):
    if target == "smallest":
        return np.argsort(theta, kind="stable")
    return np.argsort(-theta, kind="stable")


def gdk_rr(op, L, k, b, target, max_basis, min_restart, V0, precond, conv, norm_op,
           u_s=EPS, max_matvecs=10**9, mv_per_col=2, rng=None, stats=None):
    """Block GD+k (locally optimal +k restart) with Rayleigh-Ritz and soft locking.

    ``conv(theta, x, wx, rnorm) -> bool`` is the convergence test (Sec. 3.2:
    user-defined criterion).  Returns (theta[k], X[L x k]) of the first k Ritz
    pairs in target order when all k pass the test at the same time.
    """
    rng = rng if rng is not None else np.random.default_rng(99)
    st = stats if stats is not None else Stats()
    V = orthonormalize(V0, None, rng)
    W = op(V)
    st.matvecs += mv_per_col * V.shape[1]
    H = V.T @ W
    H = 0.5 * (H + H.T)
    flags = np.zeros(k, dtype=bool)
    Yprev = None
    restarts_since_reset = 0
    while True:
        st.outer += 1
        g = V.shape[1]
        theta, Y = np.linalg.eigh(H)
        order = _sort_order(theta, target)
        theta, Y = theta[order], Y[:, order]
        ncand = min(k, g)
        # Block: first b not-yet-flagged Ritz pairs among the first k; flag the
        # ones that pass and pull the next candidates in their place.
        block, Xb, Rb = [], [], []
        cand = [j for j in range(ncand) if not flags[j]]
        while cand and len(block) < b:
            take, cand = cand[: b - len(block)], cand[b - len(block):]
            X = V @ Y[:, take]
            WX = W @ Y[:, take]
            R = WX - X * theta[take]
            rn = np.linalg.norm(R, axis=0)
            for c, j in enumerate(take):
                if conv(theta[j], X[:, c], WX[:, c], rn[c]):
                    flags[j] = True
                else:
                    block.append(j)
                    Xb.append(X[:, c])
                    Rb.append(R[:, c])
        if ncand == k and flags.all():
            # Verification: all k flagged; re-test all of them together.
            X = V @ Y[:, :k]
            WX = W @ Y[:, :k]
            R = WX - X * theta[:k]
            rn = np.linalg.norm(R, axis=0)
            ok = np.array([conv(theta[j], X[:, j], WX[:, j], rn[j]) for j in range(k)])
            if ok.all():
                return theta[:k], X, st
            flags = ok
            fail = [j for j in range(k) if not ok[j]][:b]
            block, Xb, Rb = fail, [X[:, j] for j in fail], [R[:, j] for j in fail]
        if not block:
            # fewer than k Ritz pairs exist yet and all of them pass: expand
            # the basis with their residuals anyway
            block = list(range(min(b, ncand)))
            X = V @ Y[:, block]
            R = W @ Y[:, block] - X * theta[block]
            Xb, Rb = list(X.T), list(R.T)
        if st.matvecs >= max_matvecs:
            st.extra["maxit"] = True
            return theta[:k], V @ Y[:, :k], st
        Rb = np.array(Rb).T
        rnb = np.linalg.norm(Rb, axis=0)
        # Reset of V and W (Sec. 3.2).
        if restarts_since_reset > 0 and rnb.min() < math.sqrt(restarts_since_reset) * norm_op * u_s:
            V = orthonormalize(V, None, rng)
            W = op(V)
            st.matvecs += mv_per_col * V.shape[1]
            H = V.T @ W
            H = 0.5 * (H + H.T)
            restarts_since_reset = 0
            Yprev = None
            st.resets += 1
            continue
        T = precond(Rb)
        Ycur = Y[:, block]
        nb = len(block)
        if g + nb > max_basis:
            # GD+k restart: keep min_restart Ritz vectors plus the previous
            # iteration's block Ritz vectors (the +k directions).
            cols = [Y[:, :min_restart]]
            if Yprev is not None:
                cols.append(Yprev)
            Z = _orth_coeff(np.hstack(cols))
            V, W = V @ Z, W @ Z
            H = Z.T @ H @ Z
            H = 0.5 * (H + H.T)
            Ycur = Z.T @ Ycur
            st.restarts += 1
            restarts_since_reset += 1
        T = orthonormalize(T, V, rng)
        WT = op(T)
        st.matvecs += mv_per_col * T.shape[1]
        Hvt = V.T @ WT
        Htt = T.T @ WT
        Htt = 0.5 * (Htt + Htt.T)
        H = np.block([[H, Hvt], [Hvt.T, Htt]])
        V = np.hstack([V, T])
        W = np.hstack([W, WT])
        Yprev = np.vstack([Ycur, np.zeros((T.shape[1], Ycur.shape[1]))])


# ----------------------------------------------------------------------------
# Stage 2 smallest: simplified refined extraction with hard locking
# ----------------------------------------------------------------------------
def gdk_refined(op, L, k, b, taus, max_basis, min_restart, V0, precond, conv, norm_op,
                u_s=EPS, max_matvecs=10**9, mv_per_col=2, rng=None, stats=None):
    """GD+k with the simplified refined extraction (Sec. 3.2).

    For the current target i the shift tau = taus[i] is constant; (B - tau I)V = QR
    is kept and extended incrementally; the refined vectors are V y for the right
    singular vectors y of R with the smallest singular values (with V orthonormal,
    ||(B - tau I) V y|| = ||R y||).  When the first refined vector passes ``conv``
    it is locked, the basis is restarted without it, and the QR is recomputed
    with the next shift.  Restart: V <- V Z and QR(R Z) = Qt Rt, Q <- Q Qt, R <- Rt.
    Returns (theta[k], X[L x k]).
    """
    rng = rng if rng is not None else np.random.default_rng(98)
    st = stats if stats is not None else Stats()
    locked = np.zeros((L, 0))
    lthetas = []

    def fresh_qr(V, W, tau):
        Qf, Rf = np.linalg.qr(W - tau * V)
        return Qf, Rf

    V = orthonormalize(V0, None, rng)
    W = op(V)
    st.matvecs += mv_per_col * V.shape[1]
    H = V.T @ W
    H = 0.5 * (H + H.T)
    i = 0
    Q, R = fresh_qr(V, W, taus[0])
    Yprev = None
    restarts_since_reset = 0
    while i < k:
        st.outer += 1
        g = V.shape[1]
        tau = taus[i]
        _, _, Vt = np.linalg.svd(R)
        Yr = Vt[::-1].T  # right singular vectors, smallest singular value first
        nb = min(b, g)
        Y = Yr[:, :nb]
        theta = np.einsum("ij,ik,kj->j", Y, H, Y)
        X = V @ Y
        WX = W @ Y
        Rres = WX - X * theta
        rn = np.linalg.norm(Rres, axis=0)
        if conv(theta[0], X[:, 0], WX[:, 0], rn[0]):
            locked = np.hstack([locked, X[:, :1]])
            lthetas.append(theta[0])
            i += 1
            if i == k:
                break
            # forced restart without the locked direction
            keep = Yr[:, 1: min(g, min_restart + 1)]
            V, W = V @ keep, W @ keep
            H = keep.T @ H @ keep
            H = 0.5 * (H + H.T)
            Q, R = fresh_qr(V, W, taus[i])
            Yprev = None
            st.restarts += 1
            restarts_since_reset += 1
            continue
        if st.matvecs >= max_matvecs:
            st.extra["maxit"] = True
            break
        if restarts_since_reset > 0 and rn.min() < math.sqrt(restarts_since_reset) * norm_op * u_s:
            V = orthonormalize(V, locked, rng)
            W = op(V)
            st.matvecs += mv_per_col * V.shape[1]
            H = V.T @ W
            H = 0.5 * (H + H.T)
            Q, R = fresh_qr(V, W, tau)
            restarts_since_reset = 0
            Yprev = None
            st.resets += 1
            continue
        T = precond(Rres)
        Ycur = Y
        if g + nb > max_basis:
            cols = [Yr[:, :min_restart]]
            if Yprev is not None:
                cols.append(Yprev)
            Z = _orth_coeff(np.hstack(cols))
            V, W = V @ Z, W @ Z
            H = Z.T @ H @ Z
            H = 0.5 * (H + H.T)
            Qt, Rt = np.linalg.qr(R @ Z)
            Q, R = Q @ Qt, Rt
            Ycur = Z.T @ Ycur
            st.restarts += 1
            restarts_since_reset += 1
        T = orthonormalize(T, np.hstack([locked, V]), rng)
        WT = op(T)
        st.matvecs += mv_per_col * T.shape[1]
        # incremental QR of (B - tau I)[V T]
        Zc = WT - tau * T
        C1 = Q.T @ Zc
        Zc = Zc - Q @ C1
        C2 = Q.T @ Zc
        Zc = Zc - Q @ C2
        Qn, Rn = np.linalg.qr(Zc)
        Q = np.hstack([Q, Qn])
        R = np.block([[R, C1 + C2], [np.zeros((Rn.shape[0], R.shape[1])), Rn]])
        Hvt = V.T @ WT
        Htt = T.T @ WT
        Htt = 0.5 * (Htt + Htt.T)
        H = np.block([[H, Hvt], [Hvt.T, Htt]])
        V = np.hstack([V, T])
        W = np.hstack([W, WT])
        Yprev = np.vstack([Ycur, np.zeros((T.shape[1], Ycur.shape[1]))])
    X = locked
    return np.array(lthetas), X, st


# ----------------------------------------------------------------------------
# Default basis sizes (Sec. 3.4) with the reading for larger k and block sizes
# ----------------------------------------------------------------------------
def default_sizes(k, b, target, stage):
    """maxBasisSize / minRestartSize: 15/6 for fewer than 10 largest, else 35/14
    (Sec. 3.4); the stage-2 smallest basis is 35 (Sec. 4.1).  Reading for larger
    k and b: minRestart = max(default, k + b), maxBasis = max(default, minRestart + 2b)."""
    if target == "largest" and k < 10 and stage == 1:
        mb, mr = 15, 6
    elif target == "largest" and k < 10:
        mb, mr = 15, 6
    else:
        mb, mr = 35, 14
    mr = max(mr, k + b)
    mb = max(mb, mr + 2 * b)
    return mb, mr


# ----------------------------------------------------------------------------
# Algorithm 1 (PHSVDS)
# ----------------------------------------------------------------------------
def phsvds(A, k, target="largest", tol=1e-10, *, b=1, V0=None, normA=0.0, precond="jacobi",
           max_basis=0, min_restart=0, max_matvecs=10**9, seed=0, stage2=True, u_stage1=EPS, polish=True,
           bj_block=32):
    """Compute the k largest or smallest singular triplets of A (Algorithm 1).

    ``u_stage1`` is the unit roundoff of a reduced-precision first phase of
    stage 1 (mixed-precision reading).  When it exceeds EPS, stage 1 runs twice
    on C: first to the floor 10 u_stage1 ||C|| that a stage 1 stored in that
    precision reaches, then, started from those Ritz vectors, to the FP64
    criterion of Algorithm 1 line 2, so that stage 2 receives the FP64 bounds
    of Sec. 3.1.  With ``polish=False`` the reduced-precision phase hands its
    vectors straight to stage 2 (the literal two-precision reading; the lower
    bound of Sec. 3.1 is then only as good as that phase's residuals).  The
    oracle computes every phase in FP64.
    """
    A = _as_csr(A)
    m, n = A.shape
    if m < n:  # use A^T A's counterpart A A^T by working on A^T (Sec. 2.1)
        res = phsvds(A.T.tocsr(), k, target, tol, b=b, V0=V0, normA=normA, precond=precond,
                     max_basis=max_basis, min_restart=min_restart, max_matvecs=max_matvecs,
                     seed=seed, stage2=stage2, u_stage1=u_stage1, polish=polish, bj_block=bj_block)
        res["U"], res["V"] = res["V"], res["U"]
        return res
    if not (1 <= k <= n):
        raise ValueError("k must be in [1, n]")
    rng = np.random.default_rng(seed)
    normA = float(normA) if normA > 0 else estimate_norm(A)
    normC = normA * normA
    delta = tol
    # --- stage 1 on C --------------------------------------------------------
    mb, mr = default_sizes(k, b, target, 1)
    mb = max_basis or mb
    mr = min_restart or mr
    if V0 is None:
        V0 = rng.standard_normal((n, b))
    colsq = np.asarray(A.multiply(A).sum(axis=0)).ravel()  # diag(A^T A)
    if precond == "jacobi" and target == "smallest":
        dinv = 1.0 / np.where(colsq > 0, colsq, 1.0)

        def prec1(R):
            return R * dinv[:, None]
    elif precond == "block_jacobi" and target == "smallest":
        Mbj = block_jacobi(A, bj_block)

        def prec1(R):
            return Mbj @ R
    else:  # largest: no preconditioner (reading)

        def prec1(R):
            return R.copy()

    def make_conv1(u):
        def conv1(theta, x, wx, rn):
            # Algorithm 1 line 2 (floor constant: see FLOOR_C)
            return rn <= max(math.sqrt(abs(theta) * normC) * delta, FLOOR_C * u * normC)
        return conv1

    opC = lambda Z: apply_C(A, Z)  # noqa: E731
    st1 = Stats()
    if u_stage1 > EPS:
        st1a = Stats()
        _, Xa, st1a = gdk_rr(opC, n, k, b, target, mb, mr, V0, prec1, make_conv1(u_stage1),
                             normC, u_stage1, max_matvecs, 2, rng, st1a)
        st1.extra["phase_a"] = st1a
        st1.matvecs += st1a.matvecs
        V0 = Xa
    if u_stage1 > EPS and not polish:
        X = Xa
    else:
        lam, X, st1 = gdk_rr(opC, n, k, b, target, mb, mr, V0, prec1, make_conv1(EPS),
                             normC, EPS, max_matvecs, 2, rng, st1)
    # Algorithm 1 line 4: Rayleigh-Ritz on the returned vectors
    X = orthonormalize(X, None, rng)
    CX = apply_C(A, X)
    st1.matvecs += 2 * X.shape[1]
    Hk = X.T @ CX
    lam, Yk = np.linalg.eigh(0.5 * (Hk + Hk.T))
    order = _sort_order(lam, target)
    lam, Yk = lam[order], Yk[:, order]
    X = X @ Yk
    CX = CX @ Yk
    rC = np.linalg.norm(CX - X * lam, axis=0)
    # Algorithm 1 line 5
    sig = np.sqrt(np.abs(lam))
    Vv = X.copy()
    Uu = (A @ Vv) / np.where(sig > 0, sig, 1.0)
    st1.matvecs += k
    rn = triplet_residuals(A, sig, Uu, Vv)
    st1.matvecs += 2 * k
    out = dict(stats1=st1, stage2_used=False, normA=normA, sigma1=sig.copy(), rC=rC)
    if (rn < normA * delta).all() or not stage2:
        return _finish(A, sig, Uu, Vv, out)
    # --- stage 2 on B ------------------------------------------------------
    L = m + n
    X0 = np.vstack([Vv, Uu]) / math.sqrt(2.0)  # Algorithm 1 line 9

    def conv2(theta, x, wx, rnB):
        # Eq. B_secondCriterion, then Eq. res on the normalised halves
        if rnB > math.sqrt(2.0) * normA * delta:
            return False
        v, u = x[:n], x[n:]
        nv, nu = np.linalg.norm(v), np.linalg.norm(u)
        if nv == 0 or nu == 0:
            return False
        v, u = v / nv, u / nu
        Av = A @ v
        s = float(u @ Av)
        r = math.sqrt(np.sum((Av - s * u) ** 2) + np.sum((A.T @ u - s * v) ** 2))
        return r < normA * delta

    def prec2(R):
        return R.copy()

    mb2, mr2 = default_sizes(k, b, target, 2)
    mb2 = max_basis or mb2
    mr2 = min_restart or mr2
    st2 = Stats()
    opB = lambda Z: apply_B(A, Z)  # noqa: E731
    if target == "largest":
        th, XB, st2 = gdk_rr(opB, L, k, b, "largest", mb2, mr2, X0, prec2, conv2, normA, EPS,
                             max_matvecs, 2, rng, st2)
    else:
        # Algorithm 1 line 15: tau_i = max(s_i - sqrt(2) ||r^C_i|| / s_i, ||A|| eps)
        taus = np.maximum(sig - math.sqrt(2.0) * rC / np.where(sig > 0, sig, 1.0), normA * EPS)
        th, XB, st2 = gdk_refined(opB, L, k, b, taus, mb2, mr2, X0, prec2, conv2, normA, EPS,
                                  max_matvecs, 2, rng, st2)
    out["stats2"] = st2
    out["stage2_used"] = True
    # Algorithm 1 line 19 with the reading sigma = u^T A v on the normalised halves
    Vv = XB[:n] / np.linalg.norm(XB[:n], axis=0)
    Uu = XB[n:] / np.linalg.norm(XB[n:], axis=0)
    sig = np.einsum("ij,ij->j", Uu, A @ Vv)
    order = _sort_order(sig, target)
    return _finish(A, sig[order], Uu[:, order], Vv[:, order], out)


def _finish(A, sig, U, V, out):
    # sign convention: the largest-magnitude entry of each v is positive
    idx = np.argmax(np.abs(V), axis=0)
    s = np.sign(V[idx, np.arange(V.shape[1])])
    s[s == 0] = 1.0
    U = U * s
    V = V * s
    out.update(sigma=np.asarray(sig, dtype=np.float64), U=U, V=V,
               rnorm=triplet_residuals(A, sig, U, V))
    return out


# ----------------------------------------------------------------------------
# Condition-number estimate (Sec. 5)
# ----------------------------------------------------------------------------
def condest(A, rel_tol: float = 0.1, *, precond="jacobi", seed=0, max_matvecs=10**9):
    """Estimate kappa(A) = sigma_max / sigma_min as in the paper's condition-number
    experiment (Sec. 5): one largest and one smallest singular value, block size
    one, stage 1 on C stopped as soon as ||r^C|| <= rel_tol |theta| (the paper
    uses rel_tol = 0.1), no stage 2.  The largest value is found first and then
    serves as ||A|| for the smallest (reading: the floor of Algorithm 1 line 2
    becomes 10 eps max(||C||, |theta|), with ||C|| unknown, i.e. |theta|, during
    the largest solve).  Each solve ends with the Rayleigh-Ritz of Algorithm 1
    line 4 on its returned vector.  Returns a dict with sigma_max, sigma_min,
    kappa, the final residual norms ||C v - lambda v|| (rC_max, rC_min) and the
    two solves' Stats."""
    A = _as_csr(A)
    if A.shape[0] < A.shape[1]:
        A = A.T.tocsr()  # same singular values (Sec. 2.1)
    n = A.shape[1]
    rng = np.random.default_rng(seed)
    opC = lambda Z: apply_C(A, Z)  # noqa: E731

    def solve(target, normC, prec):
        def conv(theta, x, wx, rn):
            lam = abs(theta)
            return rn <= max(rel_tol * lam, FLOOR_C * EPS * max(normC, lam))

        mb, mr = default_sizes(1, 1, target, 1)
        st = Stats()
        _, X, st = gdk_rr(opC, n, 1, 1, target, mb, mr, rng.standard_normal((n, 1)), prec, conv, normC, EPS,
                          max_matvecs, 2, rng, st)
        x = X[:, :1] / np.linalg.norm(X[:, :1])
        cx = apply_C(A, x)
        lam = float(x[:, 0] @ cx[:, 0])
        return math.sqrt(abs(lam)), float(np.linalg.norm(cx[:, 0] - lam * x[:, 0])), st

    s_max, r_max, st_max = solve("largest", 0.0, lambda R: R.copy())
    colsq = np.asarray(A.multiply(A).sum(axis=0)).ravel()
    if precond == "jacobi":
        dinv = 1.0 / np.where(colsq > 0, colsq, 1.0)
        prec = lambda R: R * dinv[:, None]  # noqa: E731
    else:
        prec = lambda R: R.copy()  # noqa: E731
    s_min, r_min, st_min = solve("smallest", s_max * s_max, prec)
    return dict(sigma_max=s_max, sigma_min=s_min, kappa=s_max / s_min if s_min > 0 else math.inf,
                rC_max=r_max, rC_min=r_min, stats_largest=st_max, stats_smallest=st_min)


# ----------------------------------------------------------------------------
# Block-Jacobi preconditioner on A^T A (Sec. 4)
# ----------------------------------------------------------------------------
def block_jacobi(A, bs: int) -> sp.csr_matrix:
    """M = blockdiag((C_II + delta_I I)^-1) for consecutive blocks I of bs
    columns (the last one ragged), C_II = A_I^T A_I: the paper's block Jacobi on
    A^T A.  Readings: a zero diagonal entry (an empty column of A) is replaced
    by 1, and delta_I = 1e-10 max_r (C_II)_rr keeps rank-deficient blocks
    invertible; the dense inverse is symmetrised."""
    A = _as_csr(A)
    n = A.shape[1]
    Acsc = A.tocsc()
    rows, cols, vals = [], [], []
    for g0 in range(0, n, bs):
        g1 = min(n, g0 + bs)
        AI = Acsc[:, g0:g1].toarray()
        CII = AI.T @ AI
        d = np.diag(CII).copy()
        delta = 1e-10 * d.max()
        d[d == 0] = 1.0
        np.fill_diagonal(CII, d + delta)
        Minv = np.linalg.inv(CII)
        Minv = 0.5 * (Minv + Minv.T)
        r, c = np.meshgrid(np.arange(g0, g1), np.arange(g0, g1), indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(Minv.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
