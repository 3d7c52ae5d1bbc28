"""Helpers for the GPU tests: device buffers in each storage mode via the C-ABI."""
import numpy as np

from paper_1607_01404_gb300 import binding as B


def torch_dev():
    import torch

    return torch, torch.device("cuda:0")


def alloc_block(prec, L, ld):
    torch, dev = torch_dev()
    if prec == B.PREC_F32:
        return torch.zeros(L * ld, dtype=torch.float32, device=dev)
    if prec == B.PREC_DF64:
        return torch.zeros(2 * L * ld, dtype=torch.float32, device=dev)
    return torch.zeros(L * ld, dtype=torch.float64, device=dev)


def to_device(prec, X, ld=None):
    """Row-major device block (mode storage) from a host L x c float64 array."""
    torch, dev = torch_dev()
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    L, c = X.shape
    ld = ld or c
    src = torch.from_numpy(np.ascontiguousarray(X.T)).to(dev)  # column-major L x c
    dst = alloc_block(prec, L, ld)
    B.from_f64(prec, L, c, src, L, dst, ld)
    return dst


def to_host(prec, D, L, c, ld=None, col0=0):
    torch, dev = torch_dev()
    ld = ld or c
    out = torch.zeros(c * L, dtype=torch.float64, device=dev)
    esz = 1 if prec == B.PREC_F32 or prec == B.PREC_F64 else 2
    view = D[col0 * esz:] if col0 else D
    B.to_f64(prec, L, c, view, ld, out, L)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(c, L).T.copy()


def coef_device(prec, M):
    """Row-major coefficient matrix in the mode's format on the device."""
    torch, dev = torch_dev()
    raw = B.coef_convert(prec, np.ascontiguousarray(M, dtype=np.float64))
    return torch.from_numpy(raw).to(dev)


def csr_device(A):
    """Device CSR of a workloads.CSR in every value format (+ exactness flag)."""
    torch, dev = torch_dev()
    rp = torch.from_numpy(A.rowptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(A.colidx.astype(np.int32)).to(dev)
    va = torch.from_numpy(A.vals.astype(np.float64)).to(dev)
    nnz = A.nnz
    v32 = torch.zeros(max(nnz, 1), dtype=torch.float32, device=dev)
    v32lo = torch.zeros(max(nnz, 1), dtype=torch.float32, device=dev)
    v64 = torch.zeros(max(nnz, 1), dtype=torch.float64, device=dev)
    flags = torch.zeros(4, dtype=torch.int32, device=dev)
    if nnz:
        B.csr_values(va, v32, v32lo, v64, flags)
    torch.cuda.synchronize()
    return dict(rp=rp, ci=ci, va=va, v32=v32, v32lo=v32lo, v64=v64, exact=int(flags[0].item()) == 0)
