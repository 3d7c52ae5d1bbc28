"""CPU oracle for the PHSVDS hot path (test infrastructure).

This package is a plain, slow, FP64 restatement of the paper's method
(Wu, Romero, Stathopoulos, "PRIMME_SVDS", Algorithm 1 and Sec. 3.1-3.2), written
for checking, not for speed.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product path never
does, and it shares no code with the CUDA library.

Parity status of each function is stated in its module header.
"""
from .phsvds_fp64 import (  # noqa: F401
    EPS,
    apply_B,
    apply_C,
    estimate_norm,
    orthonormalize,
    phsvds,
    spmm,
    spmm_t,
    triplet_residuals,
)
