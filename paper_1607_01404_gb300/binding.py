"""ctypes binding of the PHSVDS C-ABI (include/phsvds.h, include/phsvds_kernels.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  There is no fallback: if ``libphsvds.so`` is missing or cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libphsvds.so")

SVDS_OK = 0
SVDS_ERR_ARG = -1
SVDS_ERR_SHAPE = -2
SVDS_ERR_CSR = -3
SVDS_ERR_VALUE = -4
SVDS_ERR_NOMEM = -5
SVDS_ERR_CUDA = -6
SVDS_ERR_NUMERIC = -7
SVDS_ERR_OPERATOR = -8
SVDS_ERR_MAXIT = 1
SVDS_OP_C = 1
SVDS_OP_B = 2
SVDS_LARGEST = 0
SVDS_SMALLEST = 1
SVDS_GDPK = 0
SVDS_JDQMR = 1
SVDS_DYNAMIC = 2
SVDS_FP32 = 1
SVDS_DF64 = 3  # double-float (FP64-class, u ~ 2^-48), not native FP64
SVDS_FP64 = SVDS_DF64  # older name of SVDS_DF64
SVDS_NATIVE_FP64 = 4
SVDS_BF16 = 5
SVDS_NORMAL_AUTO = 0
SVDS_NORMAL_TWOPASS = 1
SVDS_NORMAL_EXPLICIT = 2
SVDS_PRECOND_NONE = 0
SVDS_PRECOND_JACOBI = 1
SVDS_PRECOND_LEARNED = 2
SVDS_PRECOND_BLOCKJACOBI = 3

PREC_F32, PREC_DF64, PREC_F64 = 1, 2, 3


class svds_csr(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("colidx", C.c_void_p), ("vals", C.c_void_p),
                ("on_device", C.c_int)]


class svds_opts(C.Structure):
    _fields_ = [("maxBasisSize", C.c_int), ("minRestartSize", C.c_int), ("maxBlockSize", C.c_int),
                ("method_stage1", C.c_int), ("method_stage2", C.c_int), ("stage1_precision", C.c_int),
                ("stage1_polish", C.c_int), ("precond", C.c_int), ("aNorm", C.c_double),
                ("maxMatvecs", C.c_int64), ("maxSeconds", C.c_double), ("seed", C.c_uint64),
                ("printLevel", C.c_int), ("initSize", C.c_int), ("initV", C.c_void_p),
                ("stream", C.c_void_p), ("innerMaxIt", C.c_int), ("innerRelTol", C.c_double),
                ("innerPrecision", C.c_int), ("precondParams", C.c_void_p), ("precondModel", C.c_char_p),
                ("normalOperator", C.c_int),
                ("relTol", C.c_double),
                ("precondBlockSize", C.c_int),
                ("precondStallIts", C.c_int)]


class svds_stats(C.Structure):
    _fields_ = [("matvecs_stage1", C.c_int64), ("matvecs_stage2", C.c_int64),
                ("matvecs_stage1_lowprec", C.c_int64), ("outer_stage1", C.c_int64),
                ("outer_stage2", C.c_int64), ("restarts", C.c_int64), ("resets", C.c_int64),
                ("stage2_used", C.c_int), ("aNorm", C.c_double), ("seconds_setup", C.c_double),
                ("seconds_stage1", C.c_double), ("seconds_stage2", C.c_double),
                ("seconds_total", C.c_double), ("kernel_launches", C.c_int64),
                ("seconds_host_eig", C.c_double), ("seconds_sync_wait", C.c_double), ("host_syncs", C.c_int64),
                ("inner_steps", C.c_int64), ("seconds_precond", C.c_double), ("normal_nnz", C.c_int64),
                ("seconds_output", C.c_double),
                ("outer_stage1_jdqmr", C.c_int64),
                ("precond_fallback", C.c_int),
                ("seconds_norm", C.c_double),
                ("norm_steps", C.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

# caller-supplied operator: int apply(op, rows, nb, X, ldx, Y, ldy, stream, ctx)
APPLY_FN = C.CFUNCTYPE(C.c_int, C.c_int, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                       C.c_void_p, C.c_void_p)

# exported symbol -> (restype, argtypes)
_SIGS = {
    "svds_opts_default": (C.c_int, [C.POINTER(svds_opts)]),
    "svds_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(svds_csr), C.POINTER(svds_opts)]),
    "svds_create_op": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, C.c_int64, APPLY_FN, C.c_void_p, C.c_void_p,
                                 C.POINTER(svds_opts)]),
    "svds_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.POINTER(C.c_int), C.POINTER(svds_stats)]),
    "svds_destroy": (None, [C.c_void_p]),
    "svds_condest": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "svds_strerror": (C.c_char_p, [C.c_int]),
    "svds_last_error": (C.c_char_p, []),
    "phsvds_spmm": (C.c_int, [C.c_int, C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int,
                              C.c_void_p]),
    "phsvds_spmm_bf16": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_void_p]),
    "phsvds_to_bf16": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "phsvds_spmm_dots": (C.c_int, [C.c_int, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "phsvds_spmm_dots_scratch_bytes": (C.c_size_t, [C.c_int]),
    "phsvds_block_jacobi_nnz": (C.c_int64, [C.c_int64, C.c_int]),
    "phsvds_block_jacobi": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "phsvds_ortho": (C.c_int, [C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_int,
                               C.POINTER(C.c_int), C.c_void_p]),
    "phsvds_ortho_repair": (C.c_int, [C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64,
                                      C.c_int, C.c_uint64, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_void_p]),
    "phsvds_jd_solve": (C.c_int, [C.c_int, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                  C.c_double, C.c_void_p, C.POINTER(C.c_int), C.c_void_p]),
    "phsvds_gram": (C.c_int, [C.c_int, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                              C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "phsvds_gram_scratch_bytes": (C.c_size_t, [C.c_int, C.c_int]),
    "phsvds_gram_noalloc": (C.c_int, [C.c_int, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                                      C.c_int64, C.c_int, C.c_void_p, C.c_void_p]),
    "phsvds_combine": (C.c_int, [C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]),
    "phsvds_ritz_residual": (C.c_int, [C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_int,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int,
                                       C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "phsvds_ritz_scratch_bytes": (C.c_size_t, [C.c_int]),
    "phsvds_from_f64": (C.c_int, [C.c_int, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                  C.c_void_p]),
    "phsvds_to_f64": (C.c_int, [C.c_int, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                C.c_void_p]),
    "phsvds_csr_transpose": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "phsvds_csr_transpose_work_bytes": (C.c_size_t, [C.c_int64]),
    "phsvds_csr_values": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "phsvds_coef_convert": (C.c_int, [C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
    "phsvds_host_symeig": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "phsvds_host_svd": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    # learned preconditioner (phsvds_gnn.h)
    "phsvds_gnn_num_params": (C.c_int, []),
    "phsvds_gnn_init": (C.c_int, [C.c_uint64, C.c_void_p]),
    "phsvds_gnn_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(svds_csr), C.c_void_p]),
    "phsvds_gnn_destroy": (None, [C.c_void_p]),
    "phsvds_gnn_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "phsvds_gnn_pattern": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "phsvds_gnn_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "phsvds_gnn_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                       C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "phsvds_gnn_pairs": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_uint64, C.c_void_p, C.c_void_p]),
    "phsvds_gnn_apply_c": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "phsvds_gnn_save": (C.c_int, [C.c_char_p, C.c_void_p]),
    "phsvds_gnn_load": (C.c_int, [C.c_char_p, C.c_void_p]),
    "phsvds_gnn_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                  C.c_float]),
}


def lib():
    """Load libphsvds.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1607_01404_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


class SvdsError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().svds_strerror(code).decode()
        detailed = (SVDS_ERR_CUDA, SVDS_ERR_NUMERIC, SVDS_ERR_OPERATOR)
        extra = lib().svds_last_error().decode() if code in detailed else ""
        super().__init__(f"{where}: {msg} ({code}) {extra}".strip())
        self.code = code


def _check(code: int, where: str, allow_maxit: bool = False):
    if code == SVDS_OK or (allow_maxit and code == SVDS_ERR_MAXIT):
        return code
    raise SvdsError(code, where)


def svds_opts_default() -> svds_opts:
    o = svds_opts()
    _check(lib().svds_opts_default(C.byref(o)), "svds_opts_default")
    return o


def svds_strerror(code: int) -> str:
    return lib().svds_strerror(code).decode()


@dataclass
class Handle:
    ptr: C.c_void_p
    m: int
    n: int
    _keep: tuple = ()

    def close(self):
        if self.ptr:
            lib().svds_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_opts(**kw) -> svds_opts:
    o = svds_opts_default()
    keep = []
    for k, v in kw.items():
        if k == "initV" and v is not None:
            arr = np.asfortranarray(np.asarray(v, dtype=np.float64))
            keep.append(arr)
            o.initV = arr.ctypes.data
            o.initSize = arr.shape[1] if arr.ndim == 2 else 1
        elif k == "stream":
            o.stream = v
        elif k == "precondParams" and v is not None:
            arr = np.ascontiguousarray(v, dtype=np.float32)
            keep.append(arr)
            o.precondParams = arr.ctypes.data
        elif k == "precondModel" and v is not None:
            path = os.fsencode(v)
            keep.append(path)
            o.precondModel = path
        elif v is not None:
            setattr(o, k, v)
    o._keep = keep  # keep the guesses alive until svds_create copied them
    return o


def svds_create(rowptr, colidx, vals, m: int, n: int, opts: svds_opts | None = None, on_device: bool = False) -> Handle:
    """Create a handle from CSR arrays (numpy host arrays, or torch CUDA tensors with on_device=True)."""
    if on_device:
        rp, ci, va = rowptr.data_ptr(), colidx.data_ptr(), vals.data_ptr()
        nnz = int(colidx.numel())
        keep = (rowptr, colidx, vals)
    else:
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        rp, ci, va = rowptr.ctypes.data, colidx.ctypes.data, vals.ctypes.data
        nnz = int(colidx.shape[0])
        keep = (rowptr, colidx, vals)
    A = svds_csr(m, n, nnz, rp, ci, va, 1 if on_device else 0)
    h = C.c_void_p()
    _check(lib().svds_create(C.byref(h), C.byref(A), C.byref(opts) if opts is not None else None), "svds_create")
    return Handle(h, m, n, keep)


def svds_create_op(m: int, n: int, apply, diagC=None, opts: svds_opts | None = None) -> Handle:
    """Create a handle on an m x n matrix (m >= n) given by its operators.
    apply(op, rows, nb, X_ptr, ldx, Y_ptr, ldy, stream) is a Python function on
    device pointers (row-major FP64 blocks, see svds_create_op in phsvds.h)
    returning 0 on success; diagC: optional host array of diag(A^T A)."""

    def tramp(op, rows, nb, X, ldx, Y, ldy, stream, ctx):
        try:
            return int(apply(op, rows, nb, X, ldx, Y, ldy, stream) or 0)
        except Exception:  # an exception must not cross the C frames
            return 1

    fn = APPLY_FN(tramp)
    d = None if diagC is None else np.ascontiguousarray(diagC, dtype=np.float64)
    h = C.c_void_p()
    _check(lib().svds_create_op(C.byref(h), m, n, fn, None, d.ctypes.data if d is not None else None,
                                C.byref(opts) if opts is not None else None), "svds_create_op")
    return Handle(h, m, n, (fn, tramp, apply))


def svds_solve(h: Handle, k: int, target: int, tol: float, want_vectors: bool = True, U=None, V=None):
    """Returns (sigma, U, V, rnorm, numConverged, stats dict, return code).
    U (m x k) and V (n x k) may be given as column-major float64 arrays (for
    example views of pinned host buffers); otherwise they are allocated."""
    sigma = np.zeros(k)
    rnorm = np.zeros(k)
    for X, rows in ((U, h.m), (V, h.n)):
        if X is not None and (X.dtype != np.float64 or X.shape != (rows, k) or not X.flags.f_contiguous):
            raise ValueError("output blocks must be float64, column-major, m x k and n x k")
    if want_vectors:
        U = np.zeros((h.m, k), order="F") if U is None else U
        V = np.zeros((h.n, k), order="F") if V is None else V
    nconv = C.c_int(0)
    st = svds_stats()
    rc = lib().svds_solve(h.ptr, k, target, tol, sigma.ctypes.data,
                          U.ctypes.data if U is not None else None,
                          V.ctypes.data if V is not None else None,
                          rnorm.ctypes.data, C.byref(nconv), C.byref(st))
    _check(rc, "svds_solve", allow_maxit=True)
    return sigma, U, V, rnorm, nconv.value, st.as_dict(), rc


def svds_destroy(h: Handle):
    h.close()


def condest(A, rel_tol: float = 0.1, **opts):
    """Condition-number estimate (svds_condest): dict with sigma_max, sigma_min,
    kappa, rc and the stats of the largest and the smallest solve."""
    o = make_opts(**opts)
    h = svds_create(A.rowptr, A.colidx, A.vals, A.m, A.n, o)
    try:
        smax, smin, kap = C.c_double(), C.c_double(), C.c_double()
        st = (svds_stats * 2)()
        rc = lib().svds_condest(h.ptr, rel_tol, C.byref(smax), C.byref(smin), C.byref(kap), st)
        _check(rc, "svds_condest", allow_maxit=True)
    finally:
        h.close()
    return dict(sigma_max=smax.value, sigma_min=smin.value, kappa=kap.value, rc=rc,
                stats_largest=st[0].as_dict(), stats_smallest=st[1].as_dict())


def svds(A, k: int, target: str = "largest", tol: float = 1e-10, **opts):
    """Convenience: A is a workloads.CSR (host); returns a dict like the oracle's."""
    o = make_opts(**opts)
    h = svds_create(A.rowptr, A.colidx, A.vals, A.m, A.n, o)
    try:
        tgt = SVDS_LARGEST if target == "largest" else SVDS_SMALLEST
        sigma, U, V, rnorm, nconv, stats, rc = svds_solve(h, k, tgt, tol)
    finally:
        h.close()
    return dict(sigma=sigma, U=U, V=V, rnorm=rnorm, nconv=nconv, stats=stats, rc=rc)


# ---- kernel-level wrappers (torch CUDA tensors; for parity tests) ----
def _stream(stream):
    return None if stream is None else stream


def spmm(prec, rows, cols, rowptr, colidx, v32, v32lo, v64, X, ldx, Y, ldy, b, stream=None):
    ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    nnz = int(colidx.numel())
    _check(lib().phsvds_spmm(prec, rows, cols, nnz, ptr(rowptr), ptr(colidx), ptr(v32), ptr(v32lo), ptr(v64),
                             ptr(X), ldx, ptr(Y), ldy, b, _stream(stream)), "phsvds_spmm")


def spmm_bf16(rows, cols, rowptr, colidx, v16, X, ldx, Y, ldy, b, stream=None):
    """Y = A X (FP32 vectors) with bfloat16 values of A (torch CUDA tensors)."""
    _check(lib().phsvds_spmm_bf16(rows, cols, int(colidx.numel()), rowptr.data_ptr(), colidx.data_ptr(),
                                  v16.data_ptr(), X.data_ptr(), ldx, Y.data_ptr(), ldy, b, _stream(stream)),
           "phsvds_spmm_bf16")


def spmm_dots_scratch_bytes(nb):
    return int(lib().phsvds_spmm_dots_scratch_bytes(nb))


def spmm_dots(prec, n, rowptr, colidx, v32, v32lo, v64, nb, X, ldx, W, E1, E2, dots, scratch, stream=None):
    """W = K X fused with the four dot products of a JDQMR step (torch CUDA tensors)."""
    ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    _check(lib().phsvds_spmm_dots(prec, n, int(colidx.numel()), ptr(rowptr), ptr(colidx), ptr(v32), ptr(v32lo),
                                  ptr(v64), nb, ptr(X), ldx, ptr(W), ptr(E1), ptr(E2), ptr(dots), ptr(scratch),
                                  scratch.numel() * scratch.element_size(), _stream(stream)), "phsvds_spmm_dots")


def block_jacobi_nnz(n, bs):
    return int(lib().phsvds_block_jacobi_nnz(n, bs))


def block_jacobi(n, rowptrT, colidxT, valsT, bs, rowptr, colidx, v64=None, v32=None, stream=None):
    """CSR of the block-Jacobi inverse of A^T A from the CSR of A^T (torch CUDA tensors)."""
    ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    _check(lib().phsvds_block_jacobi(n, ptr(rowptrT), ptr(colidxT), ptr(valsT), bs, ptr(rowptr), ptr(colidx),
                                     ptr(v64), ptr(v32), _stream(stream)), "phsvds_block_jacobi")


def ortho(prec, L, V, ldv, g, T, ldt, nb, stream=None):
    """In-place CGS2 + CholQR2 of T against V (device blocks); returns the breakdown status."""
    status = C.c_int(0)
    _check(lib().phsvds_ortho(prec, L, V.data_ptr(), ldv, g, T.data_ptr(), ldt, nb, C.byref(status), _stream(stream)),
           "phsvds_ortho")
    return status.value


def ortho_repair(prec, L, V, ldv, g, T, ldt, nb, seed=1, stream=None):
    """phsvds_ortho with the solver's repair of a breakdown; returns (status, replaced)."""
    status, replaced = C.c_int(0), C.c_int(0)
    _check(lib().phsvds_ortho_repair(prec, L, V.data_ptr(), ldv, g, T.data_ptr(), ldt, nb, seed, C.byref(status),
                                     C.byref(replaced), _stream(stream)), "phsvds_ortho_repair")
    return status.value, replaced.value


def jd_solve(prec, n, rowptr, colidx, v32, v32lo, v64, nb, X, Bv, eta, dinv, maxit, xi, T, stream=None):
    """JDQMR inner solve on device blocks (torch CUDA tensors); returns the steps taken."""
    ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    steps = C.c_int(0)
    _check(lib().phsvds_jd_solve(prec, n, int(colidx.numel()), ptr(rowptr), ptr(colidx), ptr(v32), ptr(v32lo),
                                 ptr(v64), nb, ptr(X), ptr(Bv), eta.ctypes.data, ptr(dinv), maxit, xi, ptr(T),
                                 C.byref(steps), _stream(stream)), "phsvds_jd_solve")
    return steps.value


def to_bf16(v32, v16, flags, stream=None):
    _check(lib().phsvds_to_bf16(int(v32.numel()), v32.data_ptr(), v16.data_ptr(), flags.data_ptr(), _stream(stream)),
           "phsvds_to_bf16")


def gram(prec, r0, r1, P, ldp, p, Q, ldq, q, G, scratch, stream=None):
    _check(lib().phsvds_gram(prec, r0, r1, P.data_ptr(), ldp, p, Q.data_ptr(), ldq, q, G.data_ptr(),
                             scratch.data_ptr(), scratch.numel() * scratch.element_size(), _stream(stream)),
           "phsvds_gram")


def gram_noalloc(prec, r0, r1, P, ldp, p, Q, ldq, q, G, stream=None):
    """phsvds_gram without caller scratch (fixed library-internal scratch; p <= 64, q <= 8)."""
    _check(lib().phsvds_gram_noalloc(prec, r0, r1, P.data_ptr(), ldp, p, Q.data_ptr(), ldq, q, G.data_ptr(),
                                     _stream(stream)), "phsvds_gram_noalloc")


def gram_scratch_bytes(p, q):
    return int(lib().phsvds_gram_scratch_bytes(p, q))


def combine(prec, L, P, ldp, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv=None, stream=None):
    _check(lib().phsvds_combine(prec, L, P.data_ptr(), ldp, p, coef.data_ptr(),
                                In.data_ptr() if In is not None else None, ldin, alpha_one, Out.data_ptr(), ldout, q,
                                Rinv.data_ptr() if Rinv is not None else None, _stream(stream)), "phsvds_combine")


def ritz_residual(prec, L, V, W, ldv, g, Y, theta, X, R, ldb, nb, norms2, scratch, stream=None):
    _check(lib().phsvds_ritz_residual(prec, L, V.data_ptr(), W.data_ptr(), ldv, g, Y.data_ptr(), theta.data_ptr(),
                                      X.data_ptr(), R.data_ptr(), ldb, nb, norms2.data_ptr(), scratch.data_ptr(),
                                      scratch.numel() * scratch.element_size(), _stream(stream)),
           "phsvds_ritz_residual")


def ritz_scratch_bytes(nb):
    return int(lib().phsvds_ritz_scratch_bytes(nb))


def from_f64(prec, L, nc, src, lds, dst, ldd, stream=None):
    _check(lib().phsvds_from_f64(prec, L, nc, src.data_ptr(), lds, dst.data_ptr(), ldd, _stream(stream)),
           "phsvds_from_f64")


def to_f64(prec, L, nc, src, lds, dst, ldd, stream=None):
    _check(lib().phsvds_to_f64(prec, L, nc, src.data_ptr(), lds, dst.data_ptr(), ldd, _stream(stream)),
           "phsvds_to_f64")


def csr_transpose(rows, cols, rowptr, colidx, vals, rowptrT, colidxT, valsT, work, stream=None):
    nnz = int(colidx.numel())
    _check(lib().phsvds_csr_transpose(rows, cols, nnz, rowptr.data_ptr(), colidx.data_ptr(), vals.data_ptr(),
                                      rowptrT.data_ptr(), colidxT.data_ptr(), valsT.data_ptr(), work.data_ptr(),
                                      work.numel() * work.element_size(), _stream(stream)), "phsvds_csr_transpose")


def csr_transpose_work_bytes(cols):
    return int(lib().phsvds_csr_transpose_work_bytes(cols))


def csr_values(vals, v32, v32lo, v64, flags, stream=None):
    _check(lib().phsvds_csr_values(int(vals.numel()), vals.data_ptr(), v32.data_ptr(), v32lo.data_ptr(),
                                   v64.data_ptr(), flags.data_ptr(), _stream(stream)), "phsvds_csr_values")


def coef_convert(prec, src: np.ndarray) -> np.ndarray:
    """Host conversion of doubles to the mode's coefficient format (returned as raw float32/float64 words)."""
    src = np.ascontiguousarray(src, dtype=np.float64).ravel()
    if prec == PREC_F32:
        out = np.zeros(src.size, dtype=np.float32)
    elif prec == PREC_DF64:
        out = np.zeros(2 * src.size, dtype=np.float32)
    else:
        out = np.zeros(src.size, dtype=np.float64)
    _check(lib().phsvds_coef_convert(prec, src.ctypes.data, src.size, out.ctypes.data), "phsvds_coef_convert")
    return out


def host_symeig(A: np.ndarray):
    A = np.asfortranarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.zeros(n)
    Z = np.zeros((n, n), order="F")
    _check(lib().phsvds_host_symeig(n, A.ctypes.data, w.ctypes.data, Z.ctypes.data), "phsvds_host_symeig")
    return w, Z


def host_svd(R: np.ndarray):
    R = np.asfortranarray(R, dtype=np.float64)
    n = R.shape[0]
    s = np.zeros(n)
    Y = np.zeros((n, n), order="F")
    _check(lib().phsvds_host_svd(n, R.ctypes.data, s.ctypes.data, Y.ctypes.data), "phsvds_host_svd")
    return s, Y


# ---- learned preconditioner ----
def gnn_num_params() -> int:
    return int(lib().phsvds_gnn_num_params())


def gnn_init(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters (float32)."""
    theta = np.zeros(gnn_num_params(), dtype=np.float32)
    _check(lib().phsvds_gnn_init(seed, theta.ctypes.data), "phsvds_gnn_init")
    return theta


def gnn_save(path, theta):
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    if theta.shape != (gnn_num_params(),):
        raise ValueError("wrong number of parameters")
    _check(lib().phsvds_gnn_save(os.fsencode(path), theta.ctypes.data), "phsvds_gnn_save")


def gnn_load(path) -> np.ndarray:
    theta = np.zeros(gnn_num_params(), dtype=np.float32)
    _check(lib().phsvds_gnn_load(os.fsencode(path), theta.ctypes.data), "phsvds_gnn_load")
    return theta


class Gnn:
    """Graph of C = A^T A on the device plus the network's forward/backward
    (argument marshalling only; every step runs in libphsvds.so)."""

    def __init__(self, rowptr, colidx, vals, m: int, n: int, stream=None):
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        A = svds_csr(m, n, int(colidx.shape[0]), rowptr.ctypes.data, colidx.ctypes.data, vals.ctypes.data, 0)
        self.ptr = C.c_void_p()
        _check(lib().phsvds_gnn_create(C.byref(self.ptr), C.byref(A), stream), "phsvds_gnn_create")
        nn, nz = C.c_int64(), C.c_int64()
        _check(lib().phsvds_gnn_shape(self.ptr, C.byref(nn), C.byref(nz)), "phsvds_gnn_shape")
        self.n, self.nnz = nn.value, nz.value
        self.np = gnn_num_params()

    def close(self):
        if self.ptr:
            lib().phsvds_gnn_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pattern(self):
        rp = np.zeros(self.n + 1, dtype=np.int32)
        ci = np.zeros(self.nnz, dtype=np.int32)
        _check(lib().phsvds_gnn_pattern(self.ptr, rp.ctypes.data, ci.ctypes.data), "phsvds_gnn_pattern")
        return rp, ci

    def _params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        if theta.shape != (self.np,):
            raise ValueError(f"expected {self.np} parameters")
        return theta

    def forward(self, theta) -> np.ndarray:
        theta = self._params(theta)
        m = np.zeros(self.nnz, dtype=np.float32)
        _check(lib().phsvds_gnn_forward(self.ptr, theta.ctypes.data, m.ctypes.data), "phsvds_gnn_forward")
        return m

    def loss_grad(self, theta, T0, X0, power_steps: int = 4, smooth_steps: int = 30):
        """Loss and gradient from the start blocks T0 (n x P) and X0 (n x Q), P, Q <= 8."""
        theta = self._params(theta)
        T0, X0 = (np.asfortranarray(a, dtype=np.float64) for a in (T0, X0))
        loss = C.c_double(0.0)
        grad = np.zeros(self.np)
        rc = lib().phsvds_gnn_loss_grad(self.ptr, theta.ctypes.data, T0.ctypes.data, T0.shape[1], power_steps,
                                        X0.ctypes.data, X0.shape[1], smooth_steps, C.byref(loss), grad.ctypes.data)
        _check(rc, "phsvds_gnn_loss_grad")
        return loss.value, grad

    def pairs(self, P: int, smooth: int, seed: int):
        """(R, T): T = smoothed seeded N(0,1) columns, R = C T (n x P, FP64)."""
        R = np.zeros((self.n, P), order="F")
        T = np.zeros((self.n, P), order="F")
        _check(lib().phsvds_gnn_pairs(self.ptr, P, smooth, seed, R.ctypes.data, T.ctypes.data), "phsvds_gnn_pairs")
        return R, T

    def apply_c(self, X):
        X = np.asfortranarray(X, dtype=np.float64)
        Y = np.zeros_like(X, order="F")
        _check(lib().phsvds_gnn_apply_c(self.ptr, X.ctypes.data, X.shape[1], Y.ctypes.data), "phsvds_gnn_apply_c")
        return Y

    def adam(self, theta, grad, m, v, step: int, lr: float):
        """In-place Adam step on float32 arrays theta, m, v."""
        grad = np.ascontiguousarray(grad, dtype=np.float64)
        for a in (theta, m, v):
            assert a.dtype == np.float32 and a.flags.c_contiguous and a.shape == (self.np,)
        _check(lib().phsvds_gnn_adam(self.ptr, theta.ctypes.data, grad.ctypes.data, m.ctypes.data, v.ctypes.data,
                                     step, lr), "phsvds_gnn_adam")
