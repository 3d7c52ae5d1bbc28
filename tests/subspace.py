"""Angles between returned singular vectors and the exact singular subspaces.

Several results are correct where singular values are multiple (a cut
multiplet at the k-th value can return any unit vector of its subspace), so
each returned (u, v) is compared with the span of the exact vectors of ITS
cluster of equal singular values: sin(angle) <= 2 ||r|| / gap (the residual
bound for an isolated cluster, gap = distance to the nearest singular value
outside the cluster), capped at 1e-8 where the gap exceeds 1e-2 ||A||.

Exact subspaces come from the closed form of the grid-difference operators
(right vectors are Kronecker products of sine vectors; the left ones follow as
A v / sigma) or from a dense SVD of a small matrix.
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle


def sin_angle(x, basis):
    """sin of the angle between vector x and the column span of the orthonormal basis."""
    x = x / np.linalg.norm(x)
    return float(np.linalg.norm(x - basis @ (basis.T @ x)))


def _bound(res, gap, normA):
    b = 2.0 * res / gap + 1e-12
    if gap > 1e-2 * normA:
        b = min(b, 1e-8)
    return b


def grid_sigma(N, dims):
    t = 4.0 * np.sin(np.arange(1, N + 1) * np.pi / (2 * (N + 1))) ** 2
    s = t[:, None] + t[None, :] if dims == 2 else t[:, None, None] + t[None, :, None] + t[None, None, :]
    return np.sort(np.sqrt(s.ravel()))


def _grid_cluster(N, dims, sigma, rel=1e-12):
    """Right singular vectors (n x mult, orthonormal) of the grid operator for
    the singular value sigma, and the distance to the nearest other value."""
    t = 4.0 * np.sin(np.arange(1, N + 1) * np.pi / (2 * (N + 1))) ** 2
    pts = np.arange(1, N + 1)
    sines = [np.sin(i * pts * np.pi / (N + 1)) for i in range(1, N + 1)]
    sines = [s / np.linalg.norm(s) for s in sines]
    members, others = [], []
    for idx in itertools.product(range(N), repeat=dims):
        s = np.sqrt(sum(t[i] for i in idx))
        (members if abs(s - sigma) <= rel * sigma else others).append((s, idx))
    gap = min(abs(s - sigma) for s, _ in others)
    cols = []
    for _, idx in members:
        v = sines[idx[0]]
        for i in idx[1:]:
            v = np.kron(v, sines[i])
        cols.append(v)
    return np.stack(cols, axis=1), gap


def check_grid_vectors(A, N, dims, r):
    """Every returned triplet of a grid-difference operator (workloads.grid_difference)
    against the closed-form singular subspace of its value."""
    S = A.to_scipy()
    normA = grid_sigma(N, dims)[-1]
    res = oracle.triplet_residuals(A, r["sigma"], r["U"], r["V"])
    worst = 0.0
    for j, sig in enumerate(r["sigma"]):
        Vc, gap = _grid_cluster(N, dims, float(sig), rel=1e-9)
        Uc = np.linalg.qr(S @ Vc)[0]
        b = _bound(res[j], gap, normA)
        sv, su = sin_angle(r["V"][:, j], Vc), sin_angle(r["U"][:, j], Uc)
        assert sv <= b and su <= b, (j, sig, sv, su, b)
        worst = max(worst, sv, su)
    return worst


def check_dense_vectors(A, r, rel=1e-9):
    """Every returned triplet of a small matrix against the subspace of the
    dense SVD's cluster of its value (values within rel ||A|| are one cluster)."""
    D = A.to_scipy().toarray()
    U, s, Vt = np.linalg.svd(D, full_matrices=False)
    normA = s[0]
    res = oracle.triplet_residuals(A, r["sigma"], r["U"], r["V"])
    worst = 0.0
    for j, sig in enumerate(r["sigma"]):
        i0 = int(np.argmin(np.abs(s - sig)))
        inc = np.abs(s - s[i0]) <= rel * normA
        gap = np.min(np.abs(s[~inc] - s[i0])) if (~inc).any() else normA
        b = _bound(res[j], gap, normA)
        sv, su = sin_angle(r["V"][:, j], Vt[inc].T), sin_angle(r["U"][:, j], U[:, inc])
        assert sv <= b and su <= b, (j, sig, sv, su, b)
        worst = max(worst, sv, su)
    return worst
