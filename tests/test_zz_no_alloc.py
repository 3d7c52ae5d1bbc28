"""The allocation-free Gram entry point gives the same results as the regular one.

Callers that cannot allocate device memory (host callbacks, allocator hooks,
plug-ins that must not touch their host application's device heap) use
phsvds_gram_noalloc, whose scratch is a fixed device array inside the library.
This file runs last so that a failure here does not hide the other tests.
"""
import numpy as np
import pytest

from paper_1607_01404_gb300 import binding as B
from paper_1607_01404_gb300 import build as BLD
from paper_1607_01404_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from gpu_util import to_device, to_host  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    BLD.build()
    B.lib()


def _case(prec, L, p, q, r0, r1, seed):
    ldp = ((p + 3) // 4) * 4
    P = wl.dense_block(L, p, seed=seed)
    Q = wl.dense_block(L, q, seed=seed + 1)
    Pd, Qd = to_device(prec, P, ld=ldp), to_device(prec, Q)
    Ps, Qs = to_host(prec, Pd, L, ldp)[:, :p], to_host(prec, Qd, L, q)
    G_ref = torch.zeros(p * q, dtype=torch.float64, device="cuda:0")
    scratch = torch.zeros(B.gram_scratch_bytes(p, q), dtype=torch.uint8, device="cuda:0")
    B.gram(prec, r0, r1, Pd, ldp, p, Qd, q, q, G_ref, scratch)
    G = torch.full((p * q,), float("nan"), dtype=torch.float64, device="cuda:0")
    B.gram_noalloc(prec, r0, r1, Pd, ldp, p, Qd, q, q, G)
    torch.cuda.synchronize()
    norm = np.abs(Ps[r0:r1]).T @ np.abs(Qs[r0:r1])
    return G.cpu().numpy().reshape(p, q), G_ref.cpu().numpy().reshape(p, q), norm


def test_gram_noalloc_matches_gram_on_two_calls_in_a_row():
    # first call: a shape that fills about half of the static scratch
    G1, R1, n1 = _case(B.PREC_DF64, 200003, 35, 8, 0, 200003, 1)
    assert np.all(np.abs(G1 - R1) <= 1e-13 * n1 + 1e-300)
    # second call: another mode and a smaller shape; the scratch keeps the
    # first call's contents, which must not leak into this result
    G2, R2, n2 = _case(B.PREC_F32, 50001, 9, 3, 17, 40000, 3)
    assert np.all(np.abs(G2 - R2) <= 1e-13 * n2 + 1e-300)


@pytest.mark.parametrize("prec", [B.PREC_F32, B.PREC_DF64, B.PREC_F64])
def test_gram_noalloc_at_the_largest_shape(prec):
    # p = 64, q = 8: the shape that sizes the array (every block's partials used)
    G, R, nrm = _case(prec, 300007, 64, 8, 5, 300001, 7)
    assert np.all(np.abs(G - R) <= 1e-13 * nrm + 1e-300)


def test_gram_noalloc_rejects_shapes_beyond_its_scratch():
    x = torch.zeros(16 * 72, dtype=torch.float64, device="cuda:0")
    G = torch.zeros(72 * 9, dtype=torch.float64, device="cuda:0")
    with pytest.raises(B.SvdsError) as e:
        B.gram_noalloc(B.PREC_F64, 0, 16, x, 72, 72, x, 72, 8, G)
    assert e.value.code == B.SVDS_ERR_ARG
    with pytest.raises(B.SvdsError) as e:  # q = 9 > 8
        B.gram_noalloc(B.PREC_F64, 0, 16, x, 72, 16, x, 72, 9, G)
    assert e.value.code == B.SVDS_ERR_ARG
