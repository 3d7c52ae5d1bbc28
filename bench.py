"""Benchmark: seconds to k singular triplets at ||r|| <= 1e-10 ||A|| (PHSVDS).

One step = one complete solve of the workload through the C-ABI: handle
creation from a device-resident CSR (transpose, value formats), the ||A||
estimate, stage 1 and, if needed, stage 2, ending with the triplets and their
residuals on the host.  The timed "chosen" form runs DYNAMIC stage 1 (GD+k or
JDQMR correction per outer iteration, FP32 inner solves), an FP32 first phase of
stage 1 with a double-float (FP64-class) polish, and the learned sparse-
approximate-inverse preconditioner (network inference inside the timed solve).

Workload: the 3D grid-difference operator [D(x)I(x)I; I(x)D(x)I; I(x)I(x)D] on a
128^3 grid (6,340,608 x 2,097,152, 12,582,912 nnz), k = 10 smallest, block 4.
Its working set is far larger than L2, so no flush is needed between steps.

Beside the timed line the JSON reports: the plain solver with the Jacobi
preconditioner in double-float and in native FP64 (JDQMR and GD+k); the end-to-
end time from pinned host buffers; the rooflines of the dominant kernel (the
FP32 Gram) and of the SpMM; the 32^2 grid with the oracle run to completion on
the host cores; the random 1e6 x 5e5 ill-conditioned matrix with stage 1 in
double-float, FP32 and bfloat16 values; none / Jacobi / learned on held-out
weighted 256^2 grids; the chosen form against the plain solvers on a weighted
96^3 grid; the condition-number estimate; the measured FP32 and FP64 GEMM rates.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "grid3d_N128"
K, TARGET, BLOCK, TOL = 10, "smallest", 4, 1e-10
METRIC = ("sec to k triplets at ||r||<=1e-10||A|| (chosen: DYNAMIC GD+k/JDQMR stage 1 with FP32 inner solves, "
          "FP32 stage-1 phase, learned preconditioner)")
MODELS = os.path.join(ROOT, "paper_1607_01404_gb300", "gnn_models")
# DRAM bytes (read + write) of one launch from ncu captures of these kernels on
# this workload (SpMM: --set full, one warm launch each; Gram: the dram__bytes
# counters, mean of two warm launches); None where the kernel changed after
# its capture
TRAFFIC = {"spmm_C": 179_408_000, "spmm_A": 292_114_000, "spmm_AT": None, "gram_tma_f32_32x4": 303_623_936}
UNIT = "s"
# FP32 operations per product of the anchored FP64-class Gram accumulation in
# the FP32 mode (fma, subtract, fma, add; issued in pairs as packed f32x2
# instructions)
GRAM_OPS = 4
# The oracle run to completion on this workload (python -m oracle.full_solve):
# its own wall time and product count; the CPU baseline of every run scales the
# oracle's measured cost per product on a bounded sample by that count
ORACLE_RECORD_REL = "oracle/records/grid3d_N128_k10_smallest.json"
ORACLE_RECORD = os.path.join(ROOT, ORACLE_RECORD_REL)


def oracle_full_count():
    """(products with A and A^T of the oracle's full solve, its record) or (None, None)."""
    try:
        with open(ORACLE_RECORD) as f:
            rec = json.load(f)
        return int(rec["matvecs_stage1"] + rec["matvecs_stage2"]), rec
    except Exception:
        return None, None


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_setup(n_gpus, backend="nccl"):
    """Replicas: one process per GPU (torchrun environment); the process group
    only carries the barrier and the max-over-ranks of the step time."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend, init_method="env://")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception as e:  # no nvidia-smi: report no clock data
            log("clock sampler unavailable:", e)
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def spmm_roofline(A, dev, torch, B, prec, b, reps=30, with_c=True):
    """Time the CSR SpMM kernels of one C = A^T A application on the workload
    with CUDA events on their stream; algorithmic bytes per launch:
    nnz (4 index + value bytes) + 4 (rows + 1) + s b (rows + cols)."""
    from paper_1607_01404_gb300 import workloads as wl  # noqa: F401

    rp = torch.from_numpy(A.rowptr).to(dev)
    ci = torch.from_numpy(A.colidx).to(dev)
    va = torch.from_numpy(A.vals).to(dev)
    nnz = A.nnz
    v32 = torch.empty(nnz, dtype=torch.float32, device=dev)
    v32lo = torch.empty(nnz, dtype=torch.float32, device=dev)
    v64 = torch.empty(nnz, dtype=torch.float64, device=dev)
    flags = torch.zeros(4, dtype=torch.int32, device=dev)
    B.csr_values(va, v32, v32lo, v64, flags)
    exact = int(flags[0].item()) == 0
    At = A.to_scipy().T.tocsr()
    At.sort_indices()
    rpT = torch.from_numpy(At.indptr.astype(np.int32)).to(dev)
    ciT = torch.from_numpy(At.indices.astype(np.int32)).to(dev)
    vaT = torch.from_numpy(At.data).to(dev)
    v32T = torch.empty(nnz, dtype=torch.float32, device=dev)
    v32loT = torch.empty(nnz, dtype=torch.float32, device=dev)
    v64T = torch.empty(nnz, dtype=torch.float64, device=dev)
    B.csr_values(vaT, v32T, v32loT, v64T, flags)
    words = 1 if prec == B.PREC_F32 else 2
    s = 4 if prec == B.PREC_F32 else 8
    X = torch.randn(A.n * b * words, dtype=torch.float32, device=dev)
    Y = torch.zeros(A.m * b * words, dtype=torch.float32, device=dev)
    W = torch.zeros(A.n * b * words, dtype=torch.float32, device=dev)
    if prec == B.PREC_DF64:
        X.view(-1, 2)[:, 1] = 0  # valid double-float words
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    lo, loT = (None, None) if exact else (v32lo, v32loT)
    vbytes = 4 if (prec != B.PREC_F64) else 8
    if prec == B.PREC_DF64 and not exact:
        vbytes = 8
    res = {}
    nnzs = {"spmm_A": nnz, "spmm_AT": nnz}
    mats = {"spmm_A": (A.m, A.n, rp, ci, v32, lo, X, Y), "spmm_AT": (A.n, A.m, rpT, ciT, v32T, loT, Y, W)}
    v64s = {"spmm_A": v64, "spmm_AT": v64T}
    if with_c:
        _explicit_c(A, dev, torch, B, X, W, nnzs, mats, v64s)
    for name, (rows, cols, r, c, vv, vl, src, dst) in mats.items():
        v64x = v64s[name]
        for _ in range(3):
            B.spmm(prec, rows, cols, r, c, vv, vl, v64x, src, b, dst, b, b, stream=sp)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            B.spmm(prec, rows, cols, r, c, vv, vl, v64x, src, b, dst, b, b, stream=sp)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        alg = nnzs[name] * (4 + vbytes) + 4 * (rows + 1) + s * b * (rows + cols)
        res[name] = {"ms": ms, "bytes": alg, "gbs": alg / (ms * 1e-3) / 1e9}
    return res


def _explicit_c(A, dev, torch, B, X, W, nnzs, mats, v64s):
    """The explicit C = A^T A (the operator of stage 1 when it is the cheaper form)."""
    S = A.to_scipy()
    Cs = (S.T @ S).tocsr()
    Cs.sort_indices()
    rpC = torch.from_numpy(Cs.indptr.astype(np.int32)).to(dev)
    ciC = torch.from_numpy(Cs.indices.astype(np.int32)).to(dev)
    vaC = torch.from_numpy(Cs.data).to(dev)
    v32C = torch.empty(Cs.nnz, dtype=torch.float32, device=dev)
    v32loC = torch.empty(Cs.nnz, dtype=torch.float32, device=dev)
    v64C = torch.empty(Cs.nnz, dtype=torch.float64, device=dev)
    flagsC = torch.zeros(4, dtype=torch.int32, device=dev)
    B.csr_values(vaC, v32C, v32loC, v64C, flagsC)
    loC = None if int(flagsC[0].item()) == 0 else v32loC
    nnzs["spmm_C"] = Cs.nnz
    mats["spmm_C"] = (A.n, A.n, rpC, ciC, v32C, loC, X, W)
    v64s["spmm_C"] = v64C


def ortho_roofline(dev, torch, B, prec, L, g, b, reps=20):
    """The two kernels of the CGS2 + CholQR2 orthogonalisation at the workload's
    sizes (basis of g columns, block of b): the Gram G = V^T T (algorithmic
    bytes L (g + b) s) and the update T <- T - V C (L (g + 2 b) s), timed with
    CUDA events on their stream."""
    words = 1 if prec == B.PREC_F32 else 2
    s = 4 if prec == B.PREC_F32 else 8
    ldv = (g + 3) // 4 * 4
    V = torch.randn(L * ldv * words, dtype=torch.float32, device=dev)
    T = torch.randn(L * b * words, dtype=torch.float32, device=dev)
    if words == 2:
        V.view(-1, 2)[:, 1] = 0
        T.view(-1, 2)[:, 1] = 0
    G = torch.zeros(g * b, dtype=torch.float64, device=dev)
    scratch = torch.zeros(B.gram_scratch_bytes(g, b), dtype=torch.uint8, device=dev)
    coef = torch.from_numpy(B.coef_convert(prec, np.full((g, b), 1e-3))).to(dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    # the Ritz kernel (X = V Y, R = W Y - X diag(theta), norms) on a second basis W,
    # and the in-place restart V <- V Z to 18 columns (Z = the first 18 columns of
    # the identity, so the values stay put over the repeated launches)
    W = torch.randn(L * ldv * words, dtype=torch.float32, device=dev)
    if words == 2:
        W.view(-1, 2)[:, 1] = 0
    Y = torch.from_numpy(B.coef_convert(prec, np.full((g, b), 1e-2))).to(dev)
    th = torch.from_numpy(B.coef_convert(prec, np.arange(1.0, b + 1))).to(dev)
    X = torch.zeros(L * b * words, dtype=torch.float32, device=dev)
    R = torch.zeros(L * b * words, dtype=torch.float32, device=dev)
    nrm = torch.zeros(b, dtype=torch.float64, device=dev)
    rscratch = torch.zeros(B.ritz_scratch_bytes(b), dtype=torch.uint8, device=dev)
    qr = 18
    Z = torch.from_numpy(B.coef_convert(prec, np.eye(g, qr))).to(dev)
    res = {}
    for name, fn, alg in (
        ("gram", lambda: B.gram(prec, 0, L, V, ldv, g, T, b, b, G, scratch, stream=sp), L * (g + b) * s),
        ("combine", lambda: B.combine(prec, L, V, ldv, g, coef, T, b, 1, T, b, b, stream=sp), L * (g + 2 * b) * s),
        ("ritz", lambda: B.ritz_residual(prec, L, V, W, ldv, g, Y, th, X, R, b, b, nrm, rscratch, stream=sp),
         L * (2 * g + 2 * b) * s),
        ("restart", lambda: B.combine(prec, L, V, ldv, g, Z, None, 0, 0, V, ldv, qr, stream=sp), L * (g + qr) * s),
    ):
        for _ in range(3):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms": ms, "bytes": alg, "gbs": alg / (ms * 1e-3) / 1e9}
    return res


def run_gpu(args, world, rank, local):
    import torch

    from paper_1607_01404_gb300 import binding as B
    from paper_1607_01404_gb300 import workloads as wl

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    B.lib()
    A, _ = wl.workload(WORKLOAD)
    rp = torch.from_numpy(A.rowptr).to(dev)
    ci = torch.from_numpy(A.colidx).to(dev)
    va = torch.from_numpy(A.vals).to(dev)
    stream = torch.cuda.Stream(dev)
    sp = stream.cuda_stream
    tgt = B.SVDS_SMALLEST if TARGET == "smallest" else B.SVDS_LARGEST

    def opts(form, seed):
        kw = dict(maxBlockSize=BLOCK, stage1_polish=1, precond=B.SVDS_PRECOND_JACOBI, seed=seed, stream=sp,
                  maxSeconds=600.0)
        if form in ("chosen", "jdqmr"):
            # chosen: the paper's stage-1 default (DYNAMIC), FP32 first phase and
            # inner solves, learned preconditioner; "jdqmr": the same with JDQMR
            # corrections at every outer iteration
            kw.update(stage1_precision=B.SVDS_FP32, method_stage1=B.SVDS_DYNAMIC, method_stage2=B.SVDS_JDQMR,
                      innerPrecision=B.SVDS_FP32, precond=B.SVDS_PRECOND_LEARNED,
                      precondModel=os.path.join(MODELS, "wgrid3d.bin"))
            if form == "jdqmr":
                kw.update(method_stage1=B.SVDS_JDQMR)
        elif form == "plain":
            kw.update(stage1_precision=B.SVDS_DF64, method_stage1=B.SVDS_JDQMR, method_stage2=B.SVDS_JDQMR,
                      innerPrecision=B.SVDS_DF64)
        elif form == "native":  # native FP64 arithmetic throughout (IEEE binary64 on the FP64 pipe)
            kw.update(stage1_precision=B.SVDS_NATIVE_FP64, method_stage1=B.SVDS_JDQMR, method_stage2=B.SVDS_JDQMR,
                      innerPrecision=B.SVDS_DF64)
        elif form == "native_gdk":
            kw.update(stage1_precision=B.SVDS_NATIVE_FP64, method_stage1=B.SVDS_GDPK, method_stage2=B.SVDS_GDPK)
        else:  # plain GD+k
            kw.update(stage1_precision=B.SVDS_DF64, method_stage1=B.SVDS_GDPK, method_stage2=B.SVDS_GDPK)
        return B.make_opts(**kw)

    def one_solve(form, seed, host_inputs=False):
        o = opts(form, seed)
        if host_inputs:
            h = B.svds_create(A.rowptr, A.colidx, A.vals, A.m, A.n, o)
        else:
            h = B.svds_create(rp, ci, va, A.m, A.n, o, on_device=True)
        try:
            out = B.svds_solve(h, K, tgt, TOL)
        finally:
            h.close()
        return out

    def timed(form, steps, seed0):
        times, stats, last = [], [], None
        for s in range(steps):
            barrier(world)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = one_solve(form, seed0 + s)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier(world)
            times.append(e0.elapsed_time(e1) / 1e3)
            stats.append(last[5])
        return times, stats, last

    log(f"[bench] rank {rank}: warmup {args.warmup}")
    for w in range(args.warmup):
        one_solve("chosen", 100 + w + 1000 * rank)
    if args.solve_only:
        # only the chosen solves (for launch lists under a profiler)
        t, st, _ = timed("chosen", args.steps, 1 + 1000 * rank)
        return dict(solve_only=True, times=t, stats=st)
    clk = ClockSampler(local)
    clk.start()
    t_chosen, st_chosen, last = timed("chosen", args.steps, 1 + 1000 * rank)
    clocks = clk.stop()
    sigma, U, V, rnorm, nconv, stats, rc = last
    exact = np.sort(np.sqrt((4 * np.sin(np.arange(1, 129) * np.pi / 258) ** 2)[:, None, None]
                            + (4 * np.sin(np.arange(1, 129) * np.pi / 258) ** 2)[None, :, None]
                            + (4 * np.sin(np.arange(1, 129) * np.pi / 258) ** 2)[None, None, :]).ravel())[:K]
    relerr = float(np.max(np.abs(sigma - exact) / exact))
    # plain FP64-class forms on the same workload
    t_plain, st_plain, lastp = timed("plain", max(1, min(args.steps, 2)), 500 + 1000 * rank)
    relerr_p = float(np.max(np.abs(lastp[0] - exact) / exact))
    t_gdk, st_gdk, lastg = timed("gdk", 1, 700 + 1000 * rank)
    relerr_g = float(np.max(np.abs(lastg[0] - exact) / exact))
    # the plain solver in native FP64 (the FP64 pipe), JDQMR and GD+k
    native = {}
    for form in ("native", "native_gdk"):
        tn, stn, lastn = timed(form, 1, 900 + 1000 * rank)
        native[form] = dict(seconds=tn[0], stats=stn[0], sigma=lastn[0], rnorm=lastn[3], nconv=lastn[4],
                            relerr=float(np.max(np.abs(lastn[0] - exact) / exact)))
    # the chosen form with JDQMR corrections at every outer iteration
    one_solve("jdqmr", 799 + 1000 * rank)  # warm-up of that form
    t_dyn, st_dyn, lastd = timed("jdqmr", max(1, min(args.steps, 2)), 800 + 1000 * rank)
    relerr_d = float(np.max(np.abs(lastd[0] - exact) / exact))
    cond = condest_runs(B, torch, stream, rp, ci, va, A, sp)
    # end to end through the public API: the CSR of A in pinned host memory is
    # copied in by svds_create, U, V, sigma and the residual norms come back
    # into pinned host buffers (all allocated before the timed steps)
    pin = dict(rp=torch.from_numpy(A.rowptr).pin_memory(), ci=torch.from_numpy(A.colidx).pin_memory(),
               va=torch.from_numpy(A.vals).pin_memory(),
               U=torch.empty((K, A.m), dtype=torch.float64).pin_memory(),
               V=torch.empty((K, A.n), dtype=torch.float64).pin_memory())
    t_e2e_all = []
    for s_ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        te0 = time.perf_counter()
        o = opts("chosen", 7 + s_ + 1000 * rank)
        h = B.svds_create(pin["rp"].numpy(), pin["ci"].numpy(), pin["va"].numpy(), A.m, A.n, o)
        try:
            oute = B.svds_solve(h, K, tgt, TOL, U=pin["U"].numpy().T, V=pin["V"].numpy().T)
        finally:
            h.close()
        torch.cuda.synchronize()
        t_e2e_all.append(time.perf_counter() - te0)
    t_e2e = statistics.mean(t_e2e_all)  # the e2e steps' total time / steps
    h2d = A.rowptr.nbytes + A.colidx.nbytes + A.vals.nbytes
    d2h = 8 * K * (A.m + A.n + 2)
    # roofline of the dominant kernel family (CSR SpMM, FP32 phase and FP64-class)
    roof32 = spmm_roofline(A, dev, torch, B, B.PREC_F32, BLOCK)
    roofdf = spmm_roofline(A, dev, torch, B, B.PREC_DF64, BLOCK)
    # orthogonalisation kernels at the solve's sizes (basis 32 columns, block 4)
    orth = {f"{nm}_{k}": v for nm, pr in (("f32", B.PREC_F32), ("df64", B.PREC_DF64))
            for k, v in ortho_roofline(dev, torch, B, pr, A.n, 32, BLOCK).items()}
    ms_step = statistics.mean(t_chosen) * 1e3  # the K timed steps' total time / K
    ms_step = max_over_ranks(ms_step, world)
    c1 = config1_report(B, wl, sp)
    c3 = config3_report(B, wl, sp, dev, torch) if not args.skip_c3 else None
    c4 = config4_report(B, wl, sp, args.c4_seeds)
    c5 = config5_report(B, wl, sp)
    fp32_peak = gemm_peak(torch, dev, torch.float32, 8192)
    fp64_peak = gemm_peak(torch, dev, torch.float64, 4096)
    return dict(times=t_chosen, stats=st_chosen, clocks=clocks, relerr=relerr, nconv=nconv, rnorm=rnorm,
                native=native, c1=c1, c3=c3, c4=c4, c5=c5, fp32_peak=fp32_peak, fp64_peak=fp64_peak, sigma=sigma,
                t_plain=t_plain, st_plain=st_plain, relerr_plain=relerr_p, t_gdk=t_gdk, st_gdk=st_gdk,
                relerr_gdk=relerr_g, t_e2e=t_e2e, h2d=h2d, d2h=d2h, t_dyn=t_dyn, st_dyn=st_dyn,
                relerr_dyn=relerr_d, cond=cond,
                roof32=roof32, roofdf=roofdf, orth=orth, ms_step=ms_step, A=A, e2e_nconv=oute[4])


def condest_runs(B, torch, stream, rp, ci, va, A, sp):
    """Condition-number estimate (Sec. 5: one largest and one smallest value,
    block 1, ||r^C|| <= 0.1 |lambda|) on the bench matrix, device-resident CSR,
    stage 1 with GD+k corrections and an FP32 first phase; kappa of the 128^3
    grid in closed form."""
    t = 4 * np.sin(np.array([1, 128]) * np.pi / 258) ** 2
    kappa = float(np.sqrt(3 * t[1]) / np.sqrt(3 * t[0]))
    out = {"kappa_exact": kappa}
    for name, m in (("gdk", B.SVDS_GDPK),):
        o = B.make_opts(stage1_precision=B.SVDS_FP32, method_stage1=m, precond=B.SVDS_PRECOND_JACOBI, stream=sp,
                        maxSeconds=300.0)
        h = B.svds_create(rp, ci, va, A.m, A.n, o, on_device=True)
        try:
            smax, smin, kap = B.C.c_double(), B.C.c_double(), B.C.c_double()
            st = (B.svds_stats * 2)()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = B.lib().svds_condest(h.ptr, 0.1, B.C.byref(smax), B.C.byref(smin), B.C.byref(kap), st)
            e1.record(stream)
            torch.cuda.synchronize()
        finally:
            h.close()
        out[name] = dict(seconds=round(e0.elapsed_time(e1) / 1e3, 4), rc=rc, kappa=kap.value,
                         rel_err=round(abs(kap.value / kappa - 1), 5),
                         matvecs=int(st[0].matvecs_stage1 + st[1].matvecs_stage1))
    return out


def _host_residuals(S, sigma, U, V):
    """Eq. (res) recomputed on the host in FP64 from the returned vectors."""
    AV = S @ V
    AtU = S.T @ U
    return np.sqrt(np.sum((AV - U * sigma) ** 2, axis=0) + np.sum((AtU - V * sigma) ** 2, axis=0))


def _grid2d_angles(N, sigma, V, rel=1e-9):
    """sin of the angle between each returned v and the closed-form right
    singular subspace of its value (Kronecker products of sine vectors)."""
    t = 4.0 * np.sin(np.arange(1, N + 1) * np.pi / (2 * (N + 1))) ** 2
    sv = np.sqrt(t[:, None] + t[None, :])
    pts = np.arange(1, N + 1)
    sines = np.array([np.sin(i * pts * np.pi / (N + 1)) for i in range(1, N + 1)])
    sines /= np.linalg.norm(sines, axis=1, keepdims=True)
    out = []
    for j, s_ in enumerate(sigma):
        ii, jj = np.nonzero(np.abs(sv - s_) <= rel * s_)
        basis = np.stack([np.kron(sines[i], sines[k]) for i, k in zip(ii, jj)], axis=1)
        x = V[:, j] / np.linalg.norm(V[:, j])
        out.append(float(np.linalg.norm(x - basis @ (basis.T @ x))))
    return out


def _solve_timed(B, torch, A, k, target, stream, on_device=None, **kw):
    """One solve (handle creation included) timed with CUDA events on its stream."""
    o = B.make_opts(stream=stream.cuda_stream, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    if on_device is not None:
        h = B.svds_create(*on_device, A.m, A.n, o, on_device=True)
    else:
        h = B.svds_create(A.rowptr, A.colidx, A.vals, A.m, A.n, o)
    try:
        out = B.svds_solve(h, k, B.SVDS_SMALLEST if target == "smallest" else B.SVDS_LARGEST, TOL)
    finally:
        h.close()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, out


def config1_report(B, wl, sp):
    """The 2D grid-difference operator of 32^2 (2112 x 1024), the 5 smallest and
    the 5 largest triplets with block 1 (the paper's default), plain FP64
    (native and double-float GD+k, Jacobi): GPU times, sigma against the
    closed form, sin angles to the closed-form subspaces (the 5th value of
    each end is double and cut at k = 5, so its vector may lie anywhere in the
    plane), and the oracle run to completion on the host cores."""
    import torch

    A = wl.grid_difference(32, 2)
    S = A.to_scipy()
    t = 4.0 * np.sin(np.arange(1, 33) * np.pi / 66) ** 2
    sv = np.sort(np.sqrt(t[:, None] + t[None, :]).ravel())
    stream = torch.cuda.Stream()
    out = {}
    for target in ("smallest", "largest"):
        ex = sv[:5] if target == "smallest" else sv[::-1][:5]
        row = {}
        for name, prec in (("native_fp64", B.SVDS_NATIVE_FP64), ("df64", B.SVDS_DF64)):
            _solve_timed(B, torch, A, 5, target, stream, maxBlockSize=1, stage1_precision=prec,
                         initV=wl.start_block(A.n, 1, 0))  # warm
            secs, (sig, U, V, rn, nconv, st, rc) = _solve_timed(B, torch, A, 5, target, stream, maxBlockSize=1,
                                                                  stage1_precision=prec,
                                                                  initV=wl.start_block(A.n, 1, 0))
            res = _host_residuals(S, sig, U, V)
            row[name] = dict(seconds=round(secs, 5), numConverged=nconv,
                             matvecs=int(st["matvecs_stage1"] + st["matvecs_stage2"]),
                             max_rel_sigma_err=float(np.max(np.abs(sig - ex) / ex)),
                             max_res_over_normA=float(res.max() / sv[-1]),
                             max_sin_angle=max(_grid2d_angles(32, sig, V)))
        try:  # the oracle to completion on the host cores (FP64 numpy/scipy, same start vector)
            import oracle

            t0 = time.perf_counter()
            o = oracle.phsvds(A, 5, target, TOL, b=1, V0=wl.start_block(A.n, 1, 0))
            row["oracle_cpu"] = dict(seconds=round(time.perf_counter() - t0, 4), cores=os.cpu_count(),
                                     matvecs=int(o["stats1"].matvecs + (o["stats2"].matvecs if o.get("stats2") else 0)),
                                     max_rel_sigma_err=float(np.max(np.abs(o["sigma"] - ex) / ex)))
        except Exception as e:  # reported, never required
            row["oracle_cpu"] = dict(failed=str(e))
        out[target] = row
    return out


def config3_report(B, wl, sp, dev, torch):
    """The tall ill-conditioned random matrix (1,000,000 x 500,000, 16 distinct
    rows per column, N(0,1) values, column j scaled by 10^u_j, u_j ~ U(-3, 0)),
    standing in for the least-squares matrices of Table 4: the 10 largest and
    the 10 smallest triplets (block 4, JDQMR in both stages) with stage 1 in
    the FP64-class (double-float) mode, with an FP32 first phase, and with an
    FP32 first phase on bfloat16 values; per-triplet relative sigma difference
    against the double-float run, Eq. (res) recomputed in FP64 on the host,
    and the bytes and time of the two SpMM passes (A then A^T) of one
    stage-1 operator application."""
    A, _ = wl.workload("randill_1e6x5e5")
    S = A.to_scipy()
    rp = torch.from_numpy(A.rowptr).to(dev)
    ci = torch.from_numpy(A.colidx).to(dev)
    va = torch.from_numpy(A.vals).to(dev)
    stream = torch.cuda.Stream(dev)
    out = dict(workload=f"randill_1e6x5e5 ({A.m} x {A.n}, nnz {A.nnz})")
    normA = None
    for target in ("largest", "smallest"):
        runs = {}
        for name, prec in (("df64", B.SVDS_DF64), ("fp32", B.SVDS_FP32), ("bf16", B.SVDS_BF16)):
            kw = dict(maxBlockSize=4, stage1_precision=prec, method_stage1=B.SVDS_JDQMR,
                      method_stage2=B.SVDS_JDQMR, precond=B.SVDS_PRECOND_JACOBI, seed=5, maxSeconds=300.0)
            secs, (sig, U, V, rn, nconv, st, rc) = _solve_timed(B, torch, A, 10, target, stream,
                                                                  on_device=(rp, ci, va), **kw)
            normA = normA or st["aNorm"]
            res = _host_residuals(S, sig, U, V)
            runs[name] = dict(seconds=round(secs, 4), numConverged=nconv, rc=rc,
                              matvecs=int(st["matvecs_stage1"] + st["matvecs_stage2"]),
                              matvecs_lowprec=int(st["matvecs_stage1_lowprec"]), stage2_used=st["stage2_used"],
                              normal_nnz=int(st["normal_nnz"]), sigma=[float(x) for x in sig],
                              max_res_over_normA=float(res.max() / st["aNorm"]))
        ref = np.array(runs["df64"]["sigma"])
        for name in ("fp32", "bf16"):
            runs[name]["rel_sigma_diff_vs_df64"] = [float(x) for x in np.abs(np.array(runs[name]["sigma"]) - ref) / ref]
        out[target] = runs
    out["spmm_two_pass_f32"] = spmm_roofline(A, dev, torch, B, B.PREC_F32, 4, reps=10, with_c=False)
    return out


def config4_report(B, wl, sp, nseeds):
    """Held-out weighted 2D grids (256^2, log-normal edge weights sigma 1.5,
    seeds 10000 .. 10000 + nseeds - 1), the 10 smallest triplets, block 4, in
    the JDQMR form with FP32 inner solves and FP32 first phase: no
    preconditioner, Jacobi and the learned M (2D model); medians of the solve
    time and of the products with A and A^T over the seeds, and the largest
    relative sigma difference between the arms."""
    model = os.path.join(MODELS, "wgrid2d.bin")
    rows = {"none": [], "jacobi": [], "learned": []}
    maxdiff = 0.0
    for seed in range(10000, 10000 + nseeds):
        A = wl.weighted_grid(256, 2, seed)
        sig = {}
        for name, pc in (("none", B.SVDS_PRECOND_NONE), ("jacobi", B.SVDS_PRECOND_JACOBI),
                         ("learned", B.SVDS_PRECOND_LEARNED)):
            kw = dict(maxBlockSize=4, stage1_precision=B.SVDS_FP32, method_stage1=B.SVDS_JDQMR,
                      method_stage2=B.SVDS_JDQMR, precond=pc, seed=3, stream=sp, maxSeconds=120.0)
            if pc == B.SVDS_PRECOND_LEARNED:
                kw["precondModel"] = model
            h = B.svds_create(A.rowptr, A.colidx, A.vals, A.m, A.n, B.make_opts(**kw))
            try:
                s_, _, _, rn, nconv, st, rc = B.svds_solve(h, 10, B.SVDS_SMALLEST, TOL, want_vectors=False)
            finally:
                h.close()
            rows[name].append(dict(seconds=st["seconds_total"], matvecs=st["matvecs_stage1"] + st["matvecs_stage2"],
                                   outer=st["outer_stage1"] + st["outer_stage2"], nconv=nconv,
                                   fallback=st["precond_fallback"]))
            sig[name] = s_
        for name in ("none", "learned"):
            maxdiff = max(maxdiff, float(np.max(np.abs(sig[name] - sig["jacobi"]) / sig["jacobi"])))
    med = {k: dict(seconds=round(statistics.median(r["seconds"] for r in v), 4),
                   matvecs=int(statistics.median(r["matvecs"] for r in v)),
                   outer=int(statistics.median(r["outer"] for r in v)),
                   all_converged=all(r["nconv"] == 10 for r in v),
                   fallbacks=sum(1 for r in v if r["fallback"])) for k, v in rows.items()}
    return dict(seeds=f"10000..{10000 + nseeds - 1} ({nseeds} held-out seeds)", k=10, block=4, median=med,
                max_rel_sigma_diff_vs_jacobi=maxdiff,
                speedup_learned_vs_jacobi=round(med["jacobi"]["seconds"] / med["learned"]["seconds"], 3),
                speedup_learned_vs_none=round(med["none"]["seconds"] / med["learned"]["seconds"], 3))


def config5_report(B, wl, sp):
    """The weighted 3D grid of 96^3 (held-out seed 10000), the 20 smallest
    triplets, block 8: the chosen form (DYNAMIC stage 1 with an FP32 first
    phase and FP32 inner solves, learned M from the 3D model, double-float
    polish and stage 2) against the plain solver with the Jacobi
    preconditioner in double-float and in native FP64 (JDQMR in both stages)."""
    import torch

    A, meta = wl.workload("wgrid3d_N96")
    stream = torch.cuda.Stream()
    base = dict(maxBlockSize=8, precond=B.SVDS_PRECOND_JACOBI, seed=3, maxSeconds=300.0,
                method_stage1=B.SVDS_JDQMR, method_stage2=B.SVDS_JDQMR)
    forms = {
        "chosen": dict(base, stage1_precision=B.SVDS_FP32, method_stage1=B.SVDS_DYNAMIC, innerPrecision=B.SVDS_FP32,
                       precond=B.SVDS_PRECOND_LEARNED, precondModel=os.path.join(MODELS, "wgrid3d.bin")),
        "plain_df64": dict(base, stage1_precision=B.SVDS_DF64, innerPrecision=B.SVDS_DF64),
        "plain_native_fp64": dict(base, stage1_precision=B.SVDS_NATIVE_FP64, innerPrecision=B.SVDS_DF64),
    }
    out = dict(workload=f"wgrid3d_N96 seed 10000 ({A.m} x {A.n}, nnz {A.nnz})", k=20, block=8)
    sig = {}
    for name, kw in forms.items():
        _solve_timed(B, torch, A, 20, "smallest", stream, **kw) if name == "chosen" else None  # warm
        secs, (s_, U, V, rn, nconv, st, rc) = _solve_timed(B, torch, A, 20, "smallest", stream, **kw)
        sig[name] = s_
        out[name] = dict(seconds=round(secs, 4), numConverged=nconv, matvecs=int(st["matvecs_stage1"] + st["matvecs_stage2"]),
                         outer=int(st["outer_stage1"] + st["outer_stage2"]), fallback=st["precond_fallback"],
                         matvecs_lowprec=int(st["matvecs_stage1_lowprec"]),
                         max_rnorm_over_normA=float(np.max(rn) / st["aNorm"]))
    for name in ("chosen", "plain_native_fp64"):
        out[name]["max_rel_sigma_diff_vs_plain_df64"] = float(np.max(np.abs(sig[name] - sig["plain_df64"])
                                                                     / sig["plain_df64"]))
    out["speedup_chosen_vs_plain_df64"] = round(out["plain_df64"]["seconds"] / out["chosen"]["seconds"], 3)
    out["speedup_chosen_vs_plain_native_fp64"] = round(out["plain_native_fp64"]["seconds"] / out["chosen"]["seconds"], 3)
    return out


def gemm_peak(torch, dev, dtype, n):
    """Arithmetic throughput of cuBLAS GEMM in dtype (TF32 off for float32),
    n^3, best of 5, TFLOP/s: float32 measures the FP32 SIMT pipe (the
    denominator of the Gram's issue analysis), float64 the FP64 pipe (the
    reason the FP64-class mode is double-float)."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        a = torch.randn(n, n, device=dev, dtype=dtype)
        b = torch.randn(n, n, device=dev, dtype=dtype)
        for _ in range(2):
            torch.mm(a, b)
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.mm(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return 2 * n ** 3 / best / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def bench_config(A, gpus):
    """The workload and form of the timed solve (the same for both arms)."""
    return dict(workload=f"{WORKLOAD}: 3D grid-difference operator 128^3 ({A.m} x {A.n}, nnz {A.nnz})",
                k=K, target=TARGET, block=BLOCK, tol=TOL, precond="learned (gnn_models/wgrid3d.bin)",
                form="chosen: DYNAMIC stage 1 (GD+k or JDQMR correction per outer iteration by measured "
                     "rates; JDQMR inner QMR solves in FP32), FP32 stage-1 phase, learned SPAI preconditioner, "
                     "FP64-class outer polish/stage 2",
                l2="working set >> L2 (no flush)", parallelism=f"replicas x{gpus}")


def cpu_sample(A, seconds=15.0):
    """The oracle as it stands on a bounded sample: stage 1 (FP64, GD+k, Jacobi)
    on the same matrix, stopped after a matvec budget sized to ~`seconds`;
    returns (matvecs, wall seconds, threads)."""
    import oracle
    from paper_1607_01404_gb300 import workloads as wl

    V0 = wl.start_block(A.n, BLOCK, 0)
    # calibrate: a short run, then one sized to the time budget
    t0 = time.perf_counter()
    r = oracle.phsvds(A, K, TARGET, TOL, b=BLOCK, V0=V0, max_matvecs=40, stage2=False, normA=1.0)
    t1 = time.perf_counter() - t0
    mv1 = r["stats1"].matvecs
    budget = int(max(40, mv1 * seconds / max(t1, 1e-3)))
    t0 = time.perf_counter()
    r = oracle.phsvds(A, K, TARGET, TOL, b=BLOCK, V0=V0, max_matvecs=budget, stage2=False, normA=1.0)
    t2 = time.perf_counter() - t0
    return r["stats1"].matvecs, t2, os.cpu_count()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--c4-seeds", type=int, default=10, help="held-out seeds of the 256^2 preconditioner report")
    ap.add_argument("--skip-c3", action="store_true", help="skip the 1e6 x 5e5 random-matrix report")
    ap.add_argument("--solve-only", action="store_true",
                    help="run only the warm-up and timed chosen solves and print their times (for launch lists)")
    ap.add_argument("--kernels-only", action="store_true",
                    help="time only the SpMM kernels of the workload (no solver; used for ncu captures)")
    ap.add_argument("--kernels-workload", default=WORKLOAD,
                    help="workload of --kernels-only: grid3d_N128 (SpMM, Gram and combine) or randill_1e6x5e5 "
                         "(the two SpMM passes of its operator)")
    args = ap.parse_args()
    if args.kernels_only:
        import torch

        from paper_1607_01404_gb300 import binding as B
        from paper_1607_01404_gb300 import workloads as wl

        A, _ = wl.workload(args.kernels_workload)
        dev = torch.device("cuda", 0)
        B.lib()
        if args.kernels_workload != WORKLOAD:
            out = {"workload": args.kernels_workload,
                   "f32": spmm_roofline(A, dev, torch, B, B.PREC_F32, BLOCK, reps=args.steps, with_c=False)}
            print(json.dumps(out))
            return 0
        out = {"f32": spmm_roofline(A, dev, torch, B, B.PREC_F32, BLOCK, reps=args.steps),
               "df64": spmm_roofline(A, dev, torch, B, B.PREC_DF64, BLOCK, reps=args.steps),
               "ortho_f32": ortho_roofline(dev, torch, B, B.PREC_F32, A.n, 32, BLOCK, reps=args.steps),
               "ortho_df64": ortho_roofline(dev, torch, B, B.PREC_DF64, A.n, 32, BLOCK, reps=args.steps),
               # the narrow blocks of the solve's GD+k corrections (1 and 2 unconverged columns)
               "f32_b1": spmm_roofline(A, dev, torch, B, B.PREC_F32, 1, reps=args.steps),
               "f32_b2": spmm_roofline(A, dev, torch, B, B.PREC_F32, 2, reps=args.steps)}
        print(json.dumps(out))
        return 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    from paper_1607_01404_gb300 import workloads as wl

    if args.impl == "reference":
        # the CPU oracle is the reference arm: rank 0 only
        if rank != 0:
            return 0
        A, _ = wl.workload(WORKLOAD)
        vals = []
        for _ in range(args.warmup + args.steps):
            mv, secs, cores = cpu_sample(A, args.cpu_seconds / 2)
            vals.append((mv, secs))
        vals = vals[args.warmup:]
        per_mv = statistics.median(s / m for m, s in vals)
        full, rec = oracle_full_count()
        value = per_mv * full if full else None
        line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                    warmup=args.warmup, ms_per_step=statistics.median(s for _, s in vals) * 1e3,
                    higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                    config=bench_config(A, args.gpus),
                    cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle",
                                      sample=f"oracle stage-1 GD+k on the full matrix stopped after ~{vals[0][0]} "
                                             f"matvecs per step; seconds/matvec x {full} matvecs of the oracle's "
                                             f"own full solve ({ORACLE_RECORD_REL})",
                                      oracle_full_solve=rec),
                    e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
        print(json.dumps(line))
        return 0

    world, rank, local = dist_setup(args.gpus)
    res = run_gpu(args, world, rank, local)
    if rank != 0:
        return 0
    if res.get("solve_only"):
        print(json.dumps(dict(solve_only=True, seconds=res["times"],
                              kernel_launches=[s["kernel_launches"] for s in res["stats"]],
                              setup_s=[s["seconds_setup"] for s in res["stats"]],
                              norm_s=[s["seconds_norm"] for s in res["stats"]],
                              norm_steps=[s["norm_steps"] for s in res["stats"]])))
        return 0
    A = res["A"]
    peak, peak_kind = measured_peaks()
    # dominant kernel: the FP32 SpMM of the stage-1 operator (the explicit C
    # when the solver formed it, else the slower of the A and A^T passes)
    r32 = res["roof32"]
    if res["stats"][-1]["normal_nnz"] > 0:
        dom = "spmm_C"
    else:
        dom = "spmm_AT" if r32["spmm_AT"]["ms"] >= r32["spmm_A"]["ms"] else "spmm_A"
    achieved = r32[dom]["gbs"]
    st = res["stats"][-1]
    launches = int(sum(s["kernel_launches"] for s in res["stats"]))
    mv_plain = int(res["st_plain"][-1]["matvecs_stage1"] + res["st_plain"][-1]["matvecs_stage2"])
    mv_gdk = int(res["st_gdk"][0]["matvecs_stage1"] + res["st_gdk"][0]["matvecs_stage2"])
    cpu = None
    full, rec = oracle_full_count()
    try:
        mv, secs, cores = cpu_sample(A, args.cpu_seconds)
        per_mv = secs / mv
        count, whose = (full, f"the oracle's own full solve, {ORACLE_RECORD_REL}") if full else \
            (mv_gdk, "the GPU double-float GD+k count: no oracle record")
        cpu = dict(value=per_mv * count, unit=UNIT, cores=cores, kind="oracle",
                   sample=f"oracle (FP64 numpy/scipy) stage-1 GD+k on the full matrix for {mv} matvecs "
                          f"({secs:.1f} s); seconds/matvec x {count} matvecs of a full solve ({whose})",
                   oracle_full_solve=rec, config1=res["c1"])
    except Exception as e:  # the baseline is reported, never required
        cpu = dict(value=None, unit=UNIT, cores=os.cpu_count(), kind="oracle", sample=f"failed: {e}")
    value = res["ms_step"] / 1e3
    # dominant kernel of the chosen solve (launch list under profiles/): the
    # FP32 Gram of the projections; algorithmic bytes L (g + b) s of one launch
    # at the solve's shape (g = 32 basis columns, b = 4) over its CUDA-event time
    g32 = res["orth"]["f32_gram"]
    gprod = A.n * 32 * BLOCK
    gram_roof = dict(bound="hbm", kernel=f"k_gram_tma (FP32, Gram 32 x {BLOCK} columns, TMA-fed, FP64-class "
                                         f"anchored accumulation)", achieved=g32["gbs"], peak=peak, unit="GB/s",
                     frac=g32["gbs"] / peak, peak_kind=peak_kind, traffic=TRAFFIC.get("gram_tma_f32_32x4"),
                     bytes_per_launch=g32["bytes"], ms_per_launch=round(g32["ms"], 5),
                     fp32_issue=dict(ops_per_product=GRAM_OPS,
                                     achieved_tops=GRAM_OPS * gprod / (g32["ms"] * 1e-3) / 1e12,
                                     sgemm_measured_tflops=res["fp32_peak"],
                                     note="FP32 operations of the accumulation per second against cuBLAS SGEMM "
                                          "(TF32 off) measured in this run"))
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
        ms_per_step=res["ms_step"], higher_is_better=False, scaling="weak", vs_baseline=None,
        dtype="f32+df64", data="synthetic",
        config=bench_config(A, args.gpus),
        max_rel_sigma_err_vs_closed_form=res["relerr"], numConverged=res["nconv"],
        step_seconds=[round(t, 5) for t in res["times"]],
        plain_fp64=dict(value=statistics.mean(res["t_plain"]), unit=UNIT,
                        form="JDQMR, double-float (FP64-class, u ~ 2^-48) inner and outer, Jacobi",
                        matvecs=mv_plain, max_rel_sigma_err=res["relerr_plain"]),
        plain_native_fp64={k: dict(value=v["seconds"], unit=UNIT, numConverged=v["nconv"],
                                   form=("JDQMR" if k == "native" else "GD+k") + ", native FP64, Jacobi",
                                   matvecs=int(v["stats"]["matvecs_stage1"] + v["stats"]["matvecs_stage2"]),
                                   max_rel_sigma_err=v["relerr"],
                                   max_rel_sigma_diff_vs_chosen=float(np.max(np.abs(v["sigma"] - res["sigma"])
                                                                             / v["sigma"])),
                                   max_rnorm_over_normA=float(np.max(v["rnorm"]) / v["stats"]["aNorm"]))
                           for k, v in res["native"].items()},
        plain_fp64_gdk=dict(value=res["t_gdk"][0], unit=UNIT, form="GD+k, FP64-class, Jacobi",
                            matvecs=int(res["st_gdk"][0]["matvecs_stage1"] + res["st_gdk"][0]["matvecs_stage2"]),
                            max_rel_sigma_err=res["relerr_gdk"]),
        solve_stats=dict(norm_s=st["seconds_norm"], norm_steps=st["norm_steps"],
                         matvecs_stage1=st["matvecs_stage1"], matvecs_lowprec=st["matvecs_stage1_lowprec"],
                         matvecs_stage2=st["matvecs_stage2"], outer1=st["outer_stage1"], outer2=st["outer_stage2"],
                         inner_steps=st["inner_steps"], outer1_jdqmr=st["outer_stage1_jdqmr"],
                         stage2_used=st["stage2_used"], setup_s=st["seconds_setup"],
                         precond_s=st["seconds_precond"], host_syncs=st["host_syncs"],
                         sync_wait_s=st["seconds_sync_wait"], host_eig_s=st["seconds_host_eig"],
                         kernel_launches=st["kernel_launches"], precond_fallback=st["precond_fallback"]),
        roofline=gram_roof,
        roofline_spmm=dict(bound="hbm", kernel=f"{dom} (FP32, b={BLOCK})", achieved=achieved, peak=peak, unit="GB/s",
                      frac=achieved / peak, peak_kind=peak_kind, traffic=TRAFFIC.get(dom),
                      all={k: {kk: round(vv, 4) for kk, vv in v.items()} for k, v in
                           {**{f"f32_{a}": b for a, b in res["roof32"].items()},
                            **{f"df64_{a}": b for a, b in res["roofdf"].items()}}.items()}),
        ortho_roofline={k: dict(ms=round(v["ms"], 4), bytes=v["bytes"], gbs=round(v["gbs"], 1),
                                frac=round(v["gbs"] / peak, 4)) for k, v in res["orth"].items()},
        cpu_baseline=cpu,
        e2e=dict(value=res["t_e2e"], unit=UNIT, h2d_bytes_per_step=res["h2d"], d2h_bytes_per_step=res["d2h"],
                 numConverged=res["e2e_nconv"]),
        config1_grid2d_N32=res["c1"],
        config3_randill_1e6x5e5=res["c3"],
        config4_wgrid2d_N256=res["c4"],
        config5_wgrid3d_N96=res["c5"],
        chosen_jdqmr=dict(value=statistics.mean(res["t_dyn"]), unit=UNIT,
                          form="chosen form with JDQMR corrections at every stage-1 outer iteration",
                          outer1=int(res["st_dyn"][-1]["outer_stage1"]),
                          matvecs=int(res["st_dyn"][-1]["matvecs_stage1"] + res["st_dyn"][-1]["matvecs_stage2"]),
                          max_rel_sigma_err=res["relerr_dyn"]),
        condest=res["cond"],
        fp_rates_measured=dict(sgemm_tflops=round(res["fp32_peak"], 2), dgemm_tflops=round(res["fp64_peak"], 3),
                               note="cuBLAS SGEMM 8192^3 (TF32 off) and DGEMM 4096^3, best of 5, CUDA events"),
        gpu_launches=launches,
        clocks=res["clocks"],
    )
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
