"""The C-ABI library loads here (no GPU) and exports every declared symbol;
its constant tables are the correctly rounded values of the DCT constants."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_symbols():
    names = set()
    for h in HEADERS:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(blaz_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libblaz():
    from paper_2202_13007_gb300 import _build, blaz

    _build.build()
    return blaz.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["blaz_compress", "blaz_decompress", "blaz_add", "blaz_sub", "blaz_scale", "blaz_dot",
              "blaz_dot_rowcol", "blaz_matmul", "blaz_cmat_alloc", "blaz_cmat_free", "blaz_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(libblaz):
    from paper_2202_13007_gb300 import blaz

    for name in declared_symbols():
        assert hasattr(libblaz, name), name
        assert name in blaz.SIGNATURES, f"binding lacks {name}"


def test_library_constants_are_correctly_rounded(libblaz):
    mpmath = pytest.importorskip("mpmath")
    from paper_2202_13007_gb300 import blaz

    mpmath.mp.dps = 50
    cos_t, aa_t, kept = blaz.constants()
    alpha = [mpmath.sqrt(mpmath.mpf(1) / 8)] + [mpmath.mpf(1) / 2] * 7
    for k in range(8):
        for x in range(8):
            assert cos_t[k, x] == float(mpmath.cos((2 * x + 1) * k * mpmath.pi / 16))
            assert aa_t[k, x] == float(alpha[k] * alpha[x])
    want = [(i, j) for i in range(2) for j in range(8)] + [(i, j) for i in range(2, 8) for j in range(2)]
    assert [tuple(p) for p in kept] == want


def test_strerror_and_argument_errors_without_gpu(libblaz):
    from paper_2202_13007_gb300 import blaz

    assert libblaz.blaz_strerror(0) == b"ok"
    bad = blaz._CMatDesc(12, 8, None, None, None, None)   # 12 is not a multiple of 8
    assert libblaz.blaz_compress(None, 8, ctypes.byref(bad), None) == -1
    empty = blaz._CMatDesc(0, 16, None, None, None, None)
    assert libblaz.blaz_compress(None, 16, ctypes.byref(empty), None) == 0
    ok = blaz._CMatDesc(8, 8, None, None, None, None)
    assert libblaz.blaz_compress(None, 8, ctypes.byref(ok), None) == -2   # NULL arrays
    assert libblaz.blaz_matmul(ctypes.byref(empty), None, 0, 4, None, 4, 7, None) == -9   # bad mode


def test_integer_reciprocal_table_is_correctly_rounded():
    """Divisions by an integer (S/K of Eq. eqslope2, alpha_k/phi_k of
    Algorithm 1) use a table of RN(1/k) and Markstein's correction: each
    entry must be the correctly rounded reciprocal, which Python's IEEE
    division gives."""
    src = open(os.path.join(ROOT, "paper_2202_13007_gb300", "csrc", "exact_div.cuh")).read()
    body = src[src.index("c_rcp_k[256] = {"):]
    body = body[body.index("{") + 1:body.index("}")]
    vals = [float.fromhex(t) for t in body.replace("\n", " ").split(",") if t.strip()]
    assert len(vals) == 256
    assert all(v == 1.0 / k for k, v in zip(range(1, 257), vals))


def test_timeout_self_test_rejects_bad_limits_without_a_gpu(libblaz):
    """blaz_probe_bounded_wait validates its limit before anything reaches a
    device (BLAZ_ERR_ARG = -9)."""
    assert libblaz.blaz_probe_bounded_wait(-1, None) == -9
    assert libblaz.blaz_probe_bounded_wait(4000000001, None) == -9


def test_fp64_probe_rejects_bad_arguments_without_a_gpu(libblaz):
    """blaz_probe_fp64_rate checks its pointers (BLAZ_ERR_NULL = -2), its warp
    count and its round count (BLAZ_ERR_ARG = -9) before anything reaches a
    device."""
    import ctypes

    ops = ctypes.c_int64(0)
    fake = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    f = libblaz.blaz_probe_fp64_rate
    f.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    assert f(1, 16, None, 1 << 20, ctypes.byref(ops), None) == -2
    assert f(1, 16, fake, 1 << 20, None, None) == -2
    assert f(1, 0, fake, 1 << 20, ctypes.byref(ops), None) == -9
    assert f(1, 33, fake, 1 << 20, ctypes.byref(ops), None) == -9
    assert f(0, 16, fake, 1 << 20, ctypes.byref(ops), None) == -9
    assert f((1 << 30) + 1, 16, fake, 1 << 20, ctypes.byref(ops), None) == -9


def test_rate_entry_points_check_the_rate_without_a_gpu(libblaz):
    """The tunable-rate entry points reject r outside 1..8 (BLAZ_ERR_ARG = -9)
    before any descriptor or device check; keep(r) = 8r + (8-r)r."""
    import ctypes

    from paper_2202_13007_gb300 import blaz

    assert [libblaz.blaz_keep_count(r) for r in range(0, 10)] == [-1, 15, 28, 39, 48, 55, 60, 63, 64, -1]
    empty = blaz._CMatDesc(0, 16, None, None, None, None)
    e = ctypes.byref(empty)
    for r in (0, 9):
        assert libblaz.blaz_compress_rate(None, 16, r, e, None) == -9
        assert libblaz.blaz_decompress_rate(e, r, None, 16, None) == -9
        assert libblaz.blaz_add_rate(e, e, r, e, None) == -9
        assert libblaz.blaz_sub_rate(e, e, r, e, None) == -9
        assert libblaz.blaz_scale_rate(e, ctypes.c_double(2.0), r, e, None) == -9
        assert libblaz.blaz_cmat_alloc_rate(e, 8, 8, r, None) == -9
    for r in (1, 8):   # empty operands need no device
        assert libblaz.blaz_compress_rate(None, 16, r, e, None) == 0
        assert libblaz.blaz_add_rate(e, e, r, e, None) == 0


def test_dot_entry_points_reject_overflowing_shapes_without_a_gpu(libblaz):
    """blaz_dot and blaz_dot_noalloc run the same descriptor checks: sides
    above 2^34 (here 2^40 x 2^40, whose block count overflows int64) are
    BLAZ_ERR_SHAPE (-1) before anything reaches a device."""
    from paper_2202_13007_gb300 import blaz

    fake = ctypes.c_void_p(256)   # never dereferenced: the shape check fails first
    big = blaz._CMatDesc(1 << 40, 1 << 40, fake, fake, fake, fake)
    res = ctypes.c_void_p(256)
    assert libblaz.blaz_dot(ctypes.byref(big), ctypes.byref(big), res, None) == -1
    assert libblaz.blaz_dot_noalloc(ctypes.byref(big), ctypes.byref(big), res, None) == -1
    ok = blaz._CMatDesc(8, 8, fake, fake, fake, fake)
    assert libblaz.blaz_dot_noalloc(ctypes.byref(ok), ctypes.byref(big), res, None) == -1
    assert libblaz.blaz_dot_noalloc(ctypes.byref(ok), ctypes.byref(ok), None, None) == -2
