"""FP64 CPU oracle of the learned sparse-approximate-inverse preconditioner
(test infrastructure, never on the product path).

The paper has no learned component; this restates the design of this
repository's learned preconditioner so that the GPU forward and backward
kernels can be checked against it.  Every function is plain numpy/scipy.

* Graph: the structural sparsity pattern of C = A^T A (nodes = columns of A,
  symmetric, diagonal included; entries that cancel numerically are kept).
  deg_i = off-diagonal neighbours, E_i = sum_{j != i} |e_ij| (weighted degree).  c_ii = diagonal of C, deg_i = off-diagonal neighbours.
* Edge weights: e_ij = c_ij / sqrt(c_ii c_jj) for i != j (0 on the diagonal).
* Node features: x_i = [log c_ii - mean_j log c_jj, deg_i / max_j deg_j].
* Message passing, 4 layers of width 32:
      z^l = h^l W1_l + (E h^l) W2_l + b_l,  h^{l+1} = relu(z^l),  h^0 = x.
  The network applies the layer weights W1_l, W2_l in bfloat16 (the FP32
  master weights rounded to nearest even; see bf16_weights), biases and heads
  in FP32; this module computes with whatever parameters it is given, so the
  tests pass it bf16_weights(params).
* Heads: u_i = h_i . ws,  d_i = softplus(h_i . wd + bd),  delta_i = d_i / c_ii,
      s_ij = tanh(u_i + u_j + we e_ij + bs)   (symmetric by construction).
* M on the pattern of C:  m_ii = delta_i,
      m_ij = rho s_ij min(delta_i, delta_j) |e_ij| / max(E_i, E_j)   (i != j),
  so sum_{j != i} |m_ij| <= rho delta_i sum_j |e_ij| / E_i = rho delta_i < m_ii:
  M is symmetric, strictly diagonally dominant with a positive diagonal,
  hence SPD (Gershgorin).  (With s_ij = const the off-diagonal part follows
  the coupling strength |e_ij|, as a truncated Neumann series of C^-1 does.)
* Loss: a condition-number proxy of the preconditioned operator M C.  M C is
  self-adjoint in the C inner product, with Rayleigh quotient
      rho(t) = (C t)^T M (C t) / t^T C t,
  whose extremes are the extreme eigenvalues of M C.  Samples follow the
  current M: from start blocks T0 and X0,
      T = (M C)^ps T0                       (power steps: top of the spectrum),
      X = (I - omega M C)^ss X0, omega = 1 / max_p rho(t_p)   (smoothing: bottom),
      L = log mean_p rho(t_p) - log mean_q rho(x_q).
  The derivative holds T and X fixed (the Rayleigh quotient is stationary at
  eigenvectors of M C, to which the samples are driven).

Parity status: pinned by closed forms (rho of an eigenvector of C; M = I on
eigenvector samples; the power and smoothing samples converging to the
extreme eigenvalues of C for M = I), central finite differences of the
gradient with the samples fixed, scale invariance and the SPD property; the
forward pass (graph, features, every message-passing layer, both heads and M)
by a node-by-node loop restatement of the definition above on a small graph
with non-zero parameters, which separates an E/C swap, a dropped bias, a
misplaced ReLU or swapped W1/W2.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

WIDTH = 32
LAYERS = 4
RHO = 0.9


def param_shapes():
    """Ordered parameter list: (name, shape)."""
    shapes = []
    for l in range(LAYERS):
        fin = 2 if l == 0 else WIDTH
        shapes += [(f"W1_{l}", (fin, WIDTH)), (f"W2_{l}", (fin, WIDTH)), (f"b_{l}", (WIDTH,))]
    shapes += [("ws", (WIDTH,)), ("wd", (WIDTH,)), ("we", ()), ("bs", ()), ("bd", ())]
    return shapes


def n_params():
    return int(sum(int(np.prod(s)) for _, s in param_shapes()))


def unflatten(theta):
    out, o = {}, 0
    for name, shp in param_shapes():
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return out


def flatten(params):
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in param_shapes()])


def bf16_weights(params):
    """The parameters as the network applies them: W1_l and W2_l rounded to
    bfloat16 (FP32 master values, round to nearest even), the rest unchanged."""
    from .phsvds_fp64 import round_bf16

    out = dict(params)
    for name in params:
        if name.startswith("W1_") or name.startswith("W2_"):
            out[name] = round_bf16(np.asarray(params[name], dtype=np.float32)).astype(np.float64)
    return out


def init_params(seed=0):
    """Glorot-style random initialisation (seeded)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes():
        if name.startswith("W"):
            p[name] = rng.standard_normal(shp) * np.sqrt(2.0 / (shp[0] + shp[1]))
        elif name in ("ws", "wd"):
            p[name] = rng.standard_normal(shp) * np.sqrt(1.0 / WIDTH)
        elif name == "bd":
            p[name] = np.array(0.5)
        else:
            p[name] = np.zeros(shp)
    return p


class Graph:
    """Pattern of C = A^T A with the quantities the network uses."""

    def __init__(self, A):
        A = sp.csr_matrix(A)
        # structural pattern of A^T A (a product of 0/1 matrices cannot cancel)
        S = sp.csr_matrix((np.ones_like(A.data), A.indices, A.indptr), shape=A.shape)
        C = (S.T @ S).tocsr()
        C.sort_indices()
        rr = np.repeat(np.arange(C.shape[0]), np.diff(C.indptr))
        C.data = np.asarray((A.T @ A).tocsr()[rr, C.indices]).ravel().astype(np.float64)
        self.C = C
        n = C.shape[0]
        self.n = n
        self.indptr = C.indptr.astype(np.int64)
        self.indices = C.indices.astype(np.int64)
        self.cval = C.data.astype(np.float64)
        diag = C.diagonal().astype(np.float64)
        diag = np.where(diag > 0, diag, 1.0)
        self.cdiag = diag
        self.rows = np.repeat(np.arange(n), np.diff(self.indptr))
        self.offdiag = self.rows != self.indices
        self.deg = np.bincount(self.rows[self.offdiag], minlength=n).astype(np.float64)
        e = np.zeros_like(self.cval)
        r, c = self.rows[self.offdiag], self.indices[self.offdiag]
        e[self.offdiag] = self.cval[self.offdiag] / np.sqrt(diag[r] * diag[c])
        self.e = e
        self.wdeg = np.bincount(self.rows, weights=np.abs(e), minlength=n)
        self.E = sp.csr_matrix((e, self.indices, self.indptr), shape=(n, n))
        lc = np.log(diag)
        dmax = max(self.deg.max(), 1.0)
        self.x0 = np.stack([lc - lc.mean(), self.deg / dmax], axis=1)


def softplus(x):
    return np.logaddexp(0.0, x)


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def forward(G: Graph, params, keep=False):
    """Values of M on the pattern of C (same order as G.indices)."""
    h = G.x0
    cache = {"h": [h], "z": []}
    for l in range(LAYERS):
        z = h @ params[f"W1_{l}"] + (G.E @ h) @ params[f"W2_{l}"] + params[f"b_{l}"]
        h = np.maximum(z, 0.0)
        cache["z"].append(z)
        cache["h"].append(h)
    u = h @ params["ws"]
    gpre = h @ params["wd"] + params["bd"]
    d = softplus(gpre)
    delta = d / G.cdiag
    r, c = G.rows, G.indices
    a = u[r] + u[c] + params["we"] * G.e + params["bs"]
    s = np.tanh(a)
    mu = np.minimum(delta[r], delta[c])
    Emax = np.maximum(G.wdeg[r], G.wdeg[c])
    wgt = np.where(Emax > 0, np.abs(G.e) / np.where(Emax > 0, Emax, 1.0), 0.0)  # |e_ij| / max(E_i, E_j)
    m = np.where(G.offdiag, RHO * s * mu * wgt, delta[r])
    if keep:
        cache.update(u=u, gpre=gpre, d=d, delta=delta, s=s, mu=mu, wgt=wgt)
        return m, cache
    return m


def M_matrix(G: Graph, m):
    return sp.csr_matrix((m, G.indices, G.indptr), shape=(G.n, G.n))


def rayleigh(G: Graph, m, T):
    """rho_p = (C t_p)^T M (C t_p) / t_p^T C t_p and R = C T."""
    M = M_matrix(G, m)
    R = G.C @ T
    return np.sum((M @ R) * R, axis=0) / np.sum(R * T, axis=0), R


def samples(G: Graph, m, T0, X0, power_steps, smooth_steps):
    """T = (M C)^ps T0 and X = (I - omega M C)^ss X0 with omega = 1 / max rho(T)."""
    M = M_matrix(G, m)
    T = np.array(T0, dtype=np.float64)
    for _ in range(power_steps):
        T = M @ (G.C @ T)
    omega = 1.0 / rayleigh(G, m, T)[0].max()
    X = np.array(X0, dtype=np.float64)
    for _ in range(smooth_steps):
        X = X - omega * (M @ (G.C @ X))
    return T, X


def loss_from_m(G: Graph, m, T, X):
    """L = log mean rho(T) - log mean rho(X) for fixed samples, and dL/dm."""
    ra, R = rayleigh(G, m, T)
    rb, Y = rayleigh(G, m, X)
    loss = float(np.log(ra.mean()) - np.log(rb.mean()))
    # d rho_p / d m_ij = r_ip r_jp / t_p^T C t_p
    ca = 1.0 / (ra.sum() * np.sum(R * T, axis=0))
    cb = -1.0 / (rb.sum() * np.sum(Y * X, axis=0))
    dm = np.einsum("kp,kp,p->k", R[G.rows], R[G.indices], ca) + np.einsum("kq,kq,q->k", Y[G.rows], Y[G.indices], cb)
    return loss, dm


def loss_and_grad(G: Graph, params, T0, X0, power_steps, smooth_steps):
    """Loss and gradient (dict like params); the samples are taken at the current M."""
    m, cache = forward(G, params, keep=True)
    T, X = samples(G, m, T0, X0, power_steps, smooth_steps)
    loss, dm = loss_from_m(G, m, T, X)
    return loss, backward(G, params, cache, dm)


def loss_fixed_samples(G: Graph, params, T, X):
    """The loss as a function of the parameters with the samples fixed."""
    return loss_from_m(G, forward(G, params), T, X)[0]


def backward(G: Graph, params, cache, dm):
    r, c = G.rows, G.indices
    off = G.offdiag
    s, mu, wgt, delta = cache["s"], cache["mu"], cache["wgt"], cache["delta"]
    n = G.n
    ddelta = np.zeros(n)
    np.add.at(ddelta, r[~off], dm[~off])
    ds = np.where(off, dm * RHO * mu * wgt, 0.0)
    dmu = np.where(off, dm * RHO * s * wgt, 0.0)
    # min(delta_i, delta_j): the gradient goes to the smaller (ties: the lower index)
    to_i = (delta[r] < delta[c]) | ((delta[r] == delta[c]) & (r < c))
    np.add.at(ddelta, r[off & to_i], dmu[off & to_i])
    np.add.at(ddelta, c[off & ~to_i], dmu[off & ~to_i])
    da = ds * (1.0 - s * s)
    du = np.zeros(n)
    np.add.at(du, r, da)
    np.add.at(du, c, da)
    grads = {}
    grads["we"] = np.array(np.sum(da * G.e))
    grads["bs"] = np.array(np.sum(da))
    dd = ddelta / G.cdiag
    dg = dd * sigmoid(cache["gpre"])
    h = cache["h"][LAYERS]
    grads["wd"] = h.T @ dg
    grads["bd"] = np.array(np.sum(dg))
    grads["ws"] = h.T @ du
    dh = np.outer(dg, params["wd"]) + np.outer(du, params["ws"])
    for l in range(LAYERS - 1, -1, -1):
        z = cache["z"][l]
        hl = cache["h"][l]
        dz = dh * (z > 0)
        Eh = G.E @ hl
        grads[f"W1_{l}"] = hl.T @ dz
        grads[f"W2_{l}"] = Eh.T @ dz
        grads[f"b_{l}"] = dz.sum(axis=0)
        dh = dz @ params[f"W1_{l}"].T + G.E.T @ (dz @ params[f"W2_{l}"].T)
    return grads
