"""Matrices of any shape (padding reading: the matrix is extended to multiples
of 8 by repeating its last row and column; results refer to the logical
entries).  The CUDA path through the C ABI against the oracle's
`*_padded` functions: compress bit for bit, decompress / dot / products
within the tolerances of the unpadded tests."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from conftest import split_bf16_tol

pytestmark = pytest.mark.gpu

SHAPES = [(13, 21), (8, 3), (5, 8), (1, 1), (29, 16), (1001, 1003), (64, 136)]


@pytest.fixture(scope="module")
def B():
    from paper_2202_13007_gb300 import _build, blaz

    _build.build()
    blaz.lib()
    torch.cuda.init()
    return blaz


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def field(rows, cols, seed):
    rng = np.random.default_rng(seed)
    i = np.arange(rows)[:, None]
    j = np.arange(cols)[None, :]
    return np.sin(i / 9.0 + rng.uniform()) * np.cos(j / 13.0) + 1e-3 * rng.standard_normal((rows, cols))


def same(g, o):
    f, s, phi, code = g.to_host()
    assert np.array_equal(phi, o.phi) and np.array_equal(code, o.code)
    assert f.tobytes() == o.f.tobytes() and s.tobytes() == o.s.tobytes()


def block_tol(oc, rows, cols):
    """1e-12 of the block scale |f| + 14 |s| sum|c| / phi, per logical entry."""
    scale = 1e-12 * (np.abs(oc.f) + 14 * np.abs(oc.s) * np.abs(oc.code.astype(np.float64)).sum(1) / oc.phi)
    t = np.repeat(np.repeat(scale.reshape(oc.rows // 8, oc.cols // 8), 8, 0), 8, 1)
    return t[:rows, :cols]


@pytest.mark.parametrize("shape", SHAPES)
def test_compress_and_decompress_any_shape(B, shape):
    rows, cols = shape
    A = field(rows, cols, rows + 7 * cols)
    g = B.compress_padded(dev(A))
    assert (g.rows, g.cols) == (O.ceil8(rows), O.ceil8(cols)) and g.shape == shape
    oc = O.compress_padded(A)
    same(g, oc)
    # the logical entries only: a sentinel-filled wider buffer keeps its border
    big = torch.full((rows + 3, cols + 5), 7.0, dtype=torch.float64, device="cuda")
    B.decompress_padded(g, out=big[1:rows + 1, 2:cols + 2])
    got = big.cpu().numpy()
    ref = O.decompress_padded(oc, rows, cols)
    assert np.all(np.abs(got[1:rows + 1, 2:cols + 2] - ref) <= block_tol(oc, rows, cols))
    inner = np.zeros(got.shape, bool)
    inner[1:rows + 1, 2:cols + 2] = True
    assert np.all(got[~inner] == 7.0)


def test_compress_from_a_strided_unaligned_view(B):
    big = field(40, 50, 3)
    tb = dev(big)
    view = tb[1:30, 1:44]                     # lda = 50, odd offset
    g = B.compress_padded(view)
    same(g, O.compress_padded(big[1:30, 1:44]))


@pytest.mark.parametrize("shape", SHAPES)
def test_dot_over_logical_entries(B, shape):
    rows, cols = shape
    A, Bm = field(rows, cols, 1 + rows), field(rows, cols, 2 + cols)
    ga, gb = B.compress_padded(dev(A)), B.compress_padded(dev(Bm))
    v = float(B.dot_padded(ga, gb).item())
    ref, absref = O.dot_padded(O.compress_padded(A), O.compress_padded(Bm), rows, cols)
    assert abs(v - ref) <= 1e-12 * absref + 1e-300


@pytest.mark.parametrize("mode", ["fp64", "split_bf16"])
@pytest.mark.parametrize("n,k,m", [(13, 21, 7), (8, 3, 5), (29, 16, 33), (200, 131, 97)])
def test_products_over_logical_entries(B, mode, n, k, m):
    A = field(n, k, n * 3 + k)
    D = W.smoothed_normal(k, m, seed=7) if k >= 5 and m >= 5 else np.random.default_rng(5).standard_normal((k, m))
    E = field(k, m, k + 11 * m)
    ga, ge = B.compress_padded(dev(A)), B.compress_padded(dev(E))
    oa, oe = O.compress_padded(A), O.compress_padded(E)
    Ah, Eh = O.decompress_padded(oa, n, k), O.decompress_padded(oe, k, m)
    tol = 1e-12 if mode == "fp64" else split_bf16_tol(O.ceil8(k))
    C = B.matmul_padded(ga, dev(D), mode=mode).cpu().numpy()
    assert B.device_status() == 0
    assert np.all(np.abs(C - O.matmul_padded(oa, D, n, k)) <= tol * (np.abs(Ah) @ np.abs(D)) + 1e-300)
    Ccc = B.matmul_cc_padded(ga, ge, mode=mode).cpu().numpy()
    assert B.device_status() == 0
    assert np.all(np.abs(Ccc - O.matmul_cc_padded(oa, oe, n, k, m)) <= tol * (np.abs(Ah) @ np.abs(Eh)) + 1e-300)


def test_blockwise_operations_and_shape_checks(B):
    rows, cols = 21, 13
    A, Bm = field(rows, cols, 8), field(rows, cols, 9)
    ga, gb = B.compress_padded(dev(A)), B.compress_padded(dev(Bm))
    oa, ob = O.compress_padded(A), O.compress_padded(Bm)
    same(B.add(ga, gb), O.add(oa, ob))
    same(B.sub(ga, gb), O.sub(oa, ob))
    same(B.scale(ga, -1.5), O.scale(oa, -1.5))
    out = torch.empty((rows, cols), dtype=torch.float64, device="cuda")
    d = ga.desc()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for r, c in ((rows + 8, cols), (rows, cols - 8), (-1, cols)):
        assert B.lib().blaz_decompress_padded(ctypes.byref(d), r, c, out.data_ptr(), cols, st) == -1
    assert B.lib().blaz_decompress_padded(ctypes.byref(d), rows, cols, out.data_ptr(), cols - 1, st) == -3
    # ragged shapes through the plain entry points are still rejected
    with pytest.raises(ValueError):
        B.compress(dev(A))
