"""Run the FP64 oracle to completion on a named workload and record it
(test and baseline infrastructure, never on the product path).

The record holds the oracle's own wall time, thread count, products with A
and A^T (the paper's matvec count), outer iterations and the returned
singular values, so that the CPU baseline of a workload too large to solve
inside every benchmark run can be scaled by the oracle's own product count.

    python -m oracle.full_solve grid3d_N128 --out oracle/records/grid3d_N128.json
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1607_01404_gb300 import workloads as wl  # noqa: E402


def run(name: str, k: int, target: str, b: int, tol: float) -> dict:
    A, _ = wl.workload(name)
    V0 = wl.start_block(A.n, b, 0)
    t0 = time.perf_counter()
    r = oracle.phsvds(A, k, target, tol, b=b, V0=V0)
    secs = time.perf_counter() - t0
    s1, s2 = r["stats1"], r.get("stats2")
    return dict(workload=name, k=k, target=target, block=b, tol=tol, seconds=secs,
                threads=os.cpu_count(), machine=platform.machine(),
                matvecs_stage1=int(s1.matvecs), matvecs_stage2=int(s2.matvecs) if s2 is not None else 0,
                outer_stage1=int(s1.outer), stage2_used=bool(r["stage2_used"]),
                sigma=[float(x) for x in r["sigma"]], rnorm=[float(x) for x in r["rnorm"]],
                normA=float(r["normA"]))


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--target", default="smallest")
    ap.add_argument("--block", type=int, default=4)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    rec = run(a.workload, a.k, a.target, a.block, a.tol)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    with open(a.out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))
    return 0


if __name__ == "__main__":
    sys.exit(main())
