"""CPU checks of the C-ABI library: it loads, exports what the headers declare,
and rejects invalid arguments before touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1607_01404_gb300 import binding as B
from paper_1607_01404_gb300 import build as BLD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    BLD.build()


def _declared():
    names = []
    for h in ("phsvds.h", "phsvds_kernels.h", "phsvds_gnn.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(svds_\w+|phsvds_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = C.CDLL(B.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(B.exported_symbols())


def test_strerror_and_defaults():
    assert B.svds_strerror(0) == "success"
    assert "CSR" in B.svds_strerror(B.SVDS_ERR_CSR)
    o = B.svds_opts_default()
    assert o.maxBlockSize == 1 and o.stage1_precision == B.SVDS_DF64 and o.precond == B.SVDS_PRECOND_JACOBI


def test_host_symeig_matches_lapack():
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 35, 64):
        M = rng.standard_normal((n, n))
        A = M + M.T
        w, Z = B.host_symeig(A)
        np.testing.assert_allclose(w, np.linalg.eigvalsh(A), atol=1e-13 * max(1, np.abs(w).max()))
        assert np.abs(Z.T @ Z - np.eye(n)).max() < 1e-13
        assert np.abs(A @ Z - Z * w).max() < 1e-13 * max(1, np.abs(w).max())


def test_host_svd_smallest_vector_accurate():
    rng = np.random.default_rng(4)
    for n in (1, 5, 30):
        R = np.triu(rng.standard_normal((n, n)))
        R[:, 0] *= 1e-9  # tiny singular value: the refined extraction needs its vector
        s, Y = B.host_svd(R)
        sr = np.linalg.svd(R, compute_uv=False)[::-1]
        np.testing.assert_allclose(s, sr, rtol=1e-12, atol=1e-15 * sr.max())
        assert np.linalg.norm(R @ Y[:, 0]) <= s[0] * (1 + 1e-10) + 1e-15 * sr.max()


def test_coef_convert_double_float_split():
    x = np.array([1.0 / 3.0, -2.5, 1e-20, 123456.789])
    out = B.coef_convert(B.PREC_DF64, x).reshape(-1, 2)
    recon = out[:, 0].astype(np.float64) + out[:, 1].astype(np.float64)
    assert np.all(np.abs(recon - x) <= 2.0 ** -47 * np.abs(x))


def _bad_csr(kind):
    rp = np.array([0, 2, 3], dtype=np.int32)
    ci = np.array([0, 1, 1], dtype=np.int32)
    va = np.array([1.0, 2.0, 3.0])
    if kind == "unsorted":
        ci = np.array([1, 0, 1], dtype=np.int32)
    elif kind == "range":
        ci = np.array([0, 5, 1], dtype=np.int32)
    elif kind == "nan":
        va = np.array([1.0, np.nan, 3.0])
    elif kind == "rowptr":
        rp = np.array([0, 2, 2], dtype=np.int32)
    return rp, ci, va


@pytest.mark.parametrize("kind,code", [("unsorted", B.SVDS_ERR_CSR), ("range", B.SVDS_ERR_CSR),
                                       ("nan", B.SVDS_ERR_VALUE), ("rowptr", B.SVDS_ERR_CSR)])
def test_create_rejects_malformed_csr_before_any_launch(kind, code):
    rp, ci, va = _bad_csr(kind)
    with pytest.raises(B.SvdsError) as e:
        B.svds_create(rp, ci, va, 2, 2)
    assert e.value.code == code


def test_create_rejects_bad_shapes_and_options():
    rp, ci, va = _bad_csr("ok")
    with pytest.raises(B.SvdsError) as e:
        B.svds_create(rp, ci, va, 0, 2)
    assert e.value.code == B.SVDS_ERR_SHAPE
    o = B.svds_opts_default()
    o.stage1_precision = 7
    with pytest.raises(B.SvdsError) as e:
        B.svds_create(rp, ci, va, 2, 2, o)
    assert e.value.code == B.SVDS_ERR_ARG


def test_gnn_init_is_seeded_and_scaled():
    a = B.gnn_init(0)
    b = B.gnn_init(0)
    c = B.gnn_init(1)
    assert a.dtype == np.float32 and a.shape == (B.gnn_num_params(),)
    np.testing.assert_array_equal(a, b)
    assert np.any(a != c)
    # first-layer W1 (2 x 32): N(0, 2/34); bd = 0.5 is the last entry
    w = B.gnn_init(7)[:64]
    assert 0.1 < w.std() < 0.4
    assert a[-1] == np.float32(0.5)


def test_gnn_save_load_roundtrip_and_rejects_bad_files(tmp_path):
    th = B.gnn_init(3)
    p = tmp_path / "m.bin"
    B.gnn_save(p, th)
    np.testing.assert_array_equal(B.gnn_load(p), th)
    raw = p.read_bytes()
    for bad in (raw[:-4], b"XXXXXXXX" + raw[8:], raw[:8] + (5).to_bytes(4, "little") + raw[12:]):
        q = tmp_path / "bad.bin"
        q.write_bytes(bad)
        with pytest.raises(B.SvdsError):
            B.gnn_load(q)
    with pytest.raises(B.SvdsError):
        B.gnn_load(tmp_path / "missing.bin")


def test_learned_precond_needs_parameters():
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([0, 1], dtype=np.int32)
    va = np.array([1.0, 2.0])
    o = B.make_opts(precond=B.SVDS_PRECOND_LEARNED)
    with pytest.raises(B.SvdsError) as e:
        B.svds_create(rp, ci, va, 2, 2, o)
    assert e.value.code == B.SVDS_ERR_ARG
    o = B.make_opts(precond=7)
    with pytest.raises(B.SvdsError):
        B.svds_create(rp, ci, va, 2, 2, o)


@pytest.mark.parametrize("field,value", [("relTol", -0.1), ("relTol", float("nan")), ("precondBlockSize", 65),
                                         ("precondBlockSize", -1), ("method_stage1", 3), ("method_stage2", 2)])
def test_create_rejects_new_option_values(field, value):
    """Option checks of the relative mode, block Jacobi and DYNAMIC (stage 1
    only) run before any device work."""
    rp, ci, va = _bad_csr("ok")
    o = B.make_opts(**{field: value})
    with pytest.raises(B.SvdsError) as e:
        B.svds_create(rp, ci, va, 2, 2, o)
    assert e.value.code == B.SVDS_ERR_ARG


def test_condest_and_kernel_entry_argument_checks():
    import ctypes as C

    L = B.lib()
    d = C.c_double()
    assert L.svds_condest(None, 0.1, C.byref(d), C.byref(d), C.byref(d), None) == B.SVDS_ERR_ARG
    assert B.block_jacobi_nnz(100, 32) == 3 * 32 * 32 + 4 * 4
    assert B.block_jacobi_nnz(64, 64) == 64 * 64 and B.block_jacobi_nnz(10, 65) == 0
    assert L.phsvds_block_jacobi(10, None, None, None, 4, None, None, None, None, None) == B.SVDS_ERR_ARG
    assert B.spmm_dots_scratch_bytes(4) >= 2048 * 4 * 4 * 8


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of svds_csr, svds_opts and svds_stats have the
    header's size and field offsets (compiled against include/phsvds.h)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [("svds_csr", B.svds_csr), ("svds_opts", B.svds_opts), ("svds_stats", B.svds_stats)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "phsvds.h"', "int main(void) {"]
    for name, py in structs:
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (line.split() for line in out if line)}
    for name, py in structs:
        assert got[(name, "sizeof")] == C.sizeof(py), name
        for f, _ in py._fields_:
            assert got[(name, f)] == getattr(py, f).offset, (name, f)
