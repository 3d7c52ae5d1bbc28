"""Caller-supplied operators (svds_create_op; Sec. 3.4: the C and B operators
may be given directly instead of the matrix).

The operator here is the library's own FP64 SpMM on device CSR copies of A and
A^T, called from a Python function through the C-ABI.  The triplets of the
operator handle must agree with those of the CSR handle on the same matrix
and with the dense SVD, for the smallest values (Jacobi from the caller's
diag(A^T A)) and the largest, in the double-float, FP32-first-phase and native
FP64 modes; the residuals Eq. (res) are recomputed on the host."""
import numpy as np
import pytest

import oracle
from paper_1607_01404_gb300 import binding as B
from paper_1607_01404_gb300 import build as BLD
from paper_1607_01404_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    BLD.build()
    B.lib()


class CsrOperator:
    """C = A^T A and B = [0 A^T; A 0] of a host CSR matrix, applied on the device."""

    def __init__(self, A, max_cols=64):
        dev = "cuda:0"
        At = A.to_scipy().T.tocsr()
        At.sort_indices()
        self.A = A
        self.rp = torch.from_numpy(A.rowptr.astype(np.int32)).to(dev)
        self.ci = torch.from_numpy(A.colidx.astype(np.int32)).to(dev)
        self.va = torch.from_numpy(A.vals.astype(np.float64)).to(dev)
        self.rpT = torch.from_numpy(At.indptr.astype(np.int32)).to(dev)
        self.ciT = torch.from_numpy(At.indices.astype(np.int32)).to(dev)
        self.vaT = torch.from_numpy(At.data.astype(np.float64)).to(dev)
        self.tmp = torch.zeros(A.m * max_cols, dtype=torch.float64, device=dev)
        self.calls = {B.SVDS_OP_C: 0, B.SVDS_OP_B: 0}

    def _spmm(self, trans, X, ldx, Y, ldy, nb, stream):
        A = self.A
        rows, cols = (A.n, A.m) if trans else (A.m, A.n)
        rp, ci, va = (self.rpT, self.ciT, self.vaT) if trans else (self.rp, self.ci, self.va)
        return B.lib().phsvds_spmm(B.PREC_F64, rows, cols, A.nnz, rp.data_ptr(), ci.data_ptr(), None, None,
                                   va.data_ptr(), X, ldx, Y, ldy, nb, stream)

    def __call__(self, op, rows, nb, X, ldx, Y, ldy, stream):
        A = self.A
        self.calls[op] += 1
        if op == B.SVDS_OP_C:
            assert rows == A.n and nb <= self.tmp.numel() // A.m
            t = self.tmp.data_ptr()
            return self._spmm(False, X, ldx, t, nb, nb, stream) or self._spmm(True, t, nb, Y, ldy, nb, stream)
        assert op == B.SVDS_OP_B and rows == A.n + A.m
        # Y[0:n] = A^T X[n:n+m], Y[n:n+m] = A X[0:n]
        return (self._spmm(True, X + A.n * ldx * 8, ldx, Y, ldy, nb, stream)
                or self._spmm(False, X, ldx, Y + A.n * ldy * 8, ldy, nb, stream))


def _dense(A):
    return np.linalg.svd(A.to_scipy().toarray(), full_matrices=False)


@pytest.mark.parametrize("prec", [B.SVDS_DF64, B.SVDS_FP32, B.SVDS_NATIVE_FP64])
@pytest.mark.parametrize("target", ["smallest", "largest"])
def test_operator_handle_matches_csr_handle(prec, target):
    A = wl.random_illconditioned(1500, 500, 16, seed=21)
    k, tol = 4, 1e-10
    tgt = B.SVDS_SMALLEST if target == "smallest" else B.SVDS_LARGEST
    kw = dict(maxBlockSize=2, stage1_precision=prec, method_stage1=B.SVDS_JDQMR,
              precond=B.SVDS_PRECOND_JACOBI if target == "smallest" else B.SVDS_PRECOND_NONE,
              maxMatvecs=600000)
    op = CsrOperator(A)
    diagC = np.asarray((A.to_scipy().multiply(A.to_scipy())).sum(axis=0)).ravel()
    h = B.svds_create_op(A.m, A.n, op, diagC=diagC, opts=B.make_opts(**kw))
    try:
        s_op, U, V, rn, nconv, st, _ = B.svds_solve(h, k, tgt, tol)
    finally:
        h.close()
    assert nconv == k and op.calls[B.SVDS_OP_C] > 0 and op.calls[B.SVDS_OP_B] > 0
    r = B.svds(A, k, target, tol, **kw)
    np.testing.assert_allclose(s_op, r["sigma"], rtol=2e-10)
    _, s, _ = _dense(A)
    ref = s[:k] if target == "largest" else s[::-1][:k]
    np.testing.assert_allclose(s_op, ref, rtol=1e-10)
    res = oracle.triplet_residuals(A, s_op, U, V)
    assert res.max() <= tol * s[0] * 1.0000001
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-8 and np.abs(U.T @ U - np.eye(k)).max() < 1e-8


def test_operator_errors():
    A = wl.random_illconditioned(300, 100, 8, seed=2)
    op = CsrOperator(A)
    opts = B.make_opts(precond=B.SVDS_PRECOND_JACOBI)
    with pytest.raises(B.SvdsError) as e:  # Jacobi needs diag(A^T A)
        B.svds_create_op(A.m, A.n, op, opts=opts)
    assert e.value.code == B.SVDS_ERR_ARG
    with pytest.raises(B.SvdsError) as e:  # wide shapes are not accepted
        B.svds_create_op(A.n, A.m, op)
    assert e.value.code == B.SVDS_ERR_SHAPE
    with pytest.raises(B.SvdsError) as e:  # no values to round to bfloat16
        B.svds_create_op(A.m, A.n, op, opts=B.make_opts(stage1_precision=B.SVDS_BF16))
    assert e.value.code == B.SVDS_ERR_ARG

    # an operator that fails stops the solve with SVDS_ERR_OPERATOR and leaves
    # the device usable
    def failing(op_, rows, nb, X, ldx, Y, ldy, stream):
        return 7

    h = B.svds_create_op(A.m, A.n, failing, opts=B.make_opts(precond=B.SVDS_PRECOND_NONE))
    try:
        with pytest.raises(B.SvdsError) as e:
            B.svds_solve(h, 2, B.SVDS_LARGEST, 1e-8)
        assert e.value.code == B.SVDS_ERR_OPERATOR
    finally:
        h.close()
    r = B.svds(A, 2, "largest", 1e-8, precond=B.SVDS_PRECOND_NONE)
    assert r["nconv"] == 2
