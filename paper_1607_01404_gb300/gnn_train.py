"""Training driver of the learned preconditioner (initialisation, forward,
backward and Adam run in libphsvds.so; this module only schedules them).

Loss: the condition-number proxy of phsvds_gnn.h, log mean rho(t) - log
mean rho(x), with rho the Rayleigh quotient of M C in the C inner product, t
driven to the top of the spectrum of M C by power steps and x to the bottom by
smoothing steps, both with the current M.  Start blocks per training matrix
(a seeded weighted-grid operator) and step:
* T0: 8 seeded N(0,1) columns;
* X0: 4 right singular vectors of the smallest singular values of A (Ritz
  vectors harvested from a solve with the plain Jacobi solver) and 4 seeded
  N(0,1) columns.

Usage: python -m paper_1607_01404_gb300.gnn_train --out model.bin
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import binding as B
from . import workloads as wl
from .build import build


def training_matrix(family: str, N: int, seed: int) -> wl.CSR:
    """One matrix of the weighted-grid family (2D or 3D) for a seed."""
    return wl.weighted_grid(N, 2 if family == "wgrid2d" else 3, seed=seed)


def harvest(A: wl.CSR, seed: int, k: int = 4):
    """Ritz vectors of one training matrix (smallest singular values, plain Jacobi solver)."""
    res = B.svds(A, k, "smallest", tol=1e-6, maxBlockSize=4, method_stage1=B.SVDS_JDQMR,
                 stage1_precision=B.SVDS_FP32, seed=seed + 1)
    return np.asfortranarray(res["V"][:, :k])


def train(family: str = "wgrid2d", N: int = 64, seeds=range(0, 32), epochs: int = 40, lr: float = 3e-3,
          init_seed: int = 0, power_steps: int = 4, smooth_steps: int = 30, log=None):
    """Adam on the training matrices in turn; returns (theta, history of mean losses per epoch)."""
    build()
    data = []
    for s in seeds:
        A = training_matrix(family, N, s)
        g = B.Gnn(A.rowptr, A.colidx, A.vals, A.m, A.n)
        data.append((g, harvest(A, s), np.random.default_rng(7919 * s + 1)))
    theta = B.gnn_init(init_seed)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    hist = []
    step = 0
    for ep in range(epochs):
        tot = 0.0
        for g, ritz, rng in data:
            T0 = rng.standard_normal((g.n, 8))
            X0 = np.hstack([ritz, rng.standard_normal((g.n, 8 - ritz.shape[1]))])
            loss, grad = g.loss_grad(theta, T0, X0, power_steps, smooth_steps)
            step += 1
            g.adam(theta, grad, m, v, step, lr)
            tot += loss
        hist.append(tot / len(data))
        if log:
            log(f"epoch {ep} mean loss {hist[-1]:.5f}")
    for g, _, _ in data:
        g.close()
    return theta, hist


def evaluate(theta, A: wl.CSR, k: int, block: int, tol: float = 1e-10, **opts):
    """Stage-1 cost of none / Jacobi / learned on one matrix (same solver otherwise)."""
    out = {}
    for name, pc in (("none", B.SVDS_PRECOND_NONE), ("jacobi", B.SVDS_PRECOND_JACOBI),
                     ("learned", B.SVDS_PRECOND_LEARNED)):
        kw = dict(opts)
        kw["precond"] = pc
        if pc == B.SVDS_PRECOND_LEARNED:
            kw["precondParams"] = theta
        r = B.svds(A, k, "smallest", tol=tol, maxBlockSize=block, **kw)
        st = r["stats"]
        out[name] = dict(sigma=r["sigma"], rnorm=r["rnorm"], nconv=r["nconv"], seconds=st["seconds_total"],
                         seconds_stage1=st["seconds_stage1"], seconds_precond=st["seconds_precond"],
                         matvecs_stage1=st["matvecs_stage1"], outer_stage1=st["outer_stage1"],
                         inner_steps=st["inner_steps"])
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--family", default="wgrid2d", choices=["wgrid2d", "wgrid3d"])
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--seeds", type=int, default=32, help="training seeds 0 .. seeds-1")
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    t0 = time.time()
    theta, hist = train(a.family, a.N, range(a.seeds), a.epochs, a.lr, log=print)
    B.gnn_save(a.out, theta)
    print(f"saved {a.out}: loss {hist[0]:.5f} -> {hist[-1]:.5f} in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
