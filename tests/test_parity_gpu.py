"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Codes, phi, f and s of compress / add / sub / scale are compared bit for bit
(NaN outputs compared as NaN).  Floating-point results use tolerances derived
from the arithmetic:
  decompress: |d| <= 1e-12 * (|f| + 14 |s| sum|c|/phi) per block (the
              recurrence adds at most 14 IDCT terms of size <= |s| sum|c|/phi);
  dot:        |d| <= 1e-12 * sum |A_hat B_hat|;
  matmul FP64:|d_ij| <= 1e-12 * (|A_hat| |B|)_ij (componentwise).
"""
import concurrent.futures as cf
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from conftest import SPLIT_BF16_LARGE_K_TOL, split_bf16_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def B():
    from paper_2202_13007_gb300 import _build, blaz

    _build.build()
    blaz.lib()
    torch.cuda.init()
    return blaz


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def same_bits(x, y):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    nan = np.isnan(x)
    assert np.array_equal(nan, np.isnan(y))
    assert np.array_equal(x[~nan].view(np.uint64), y[~nan].view(np.uint64))


def assert_cmat_equal(g, o, idx=None):
    f, s, phi, code = g.to_host()
    if idx is not None:
        f, s, phi, code = f[idx], s[idx], phi[idx], code[idx]
    assert np.array_equal(phi, o.phi if hasattr(o, "phi") else o[2])
    assert np.array_equal(code, o.code if hasattr(o, "code") else o[3])
    same_bits(f, o.f if hasattr(o, "f") else o[0])
    same_bits(s, o.s if hasattr(o, "s") else o[1])


def decompress_tol(oc):
    scale = np.abs(oc.f) + 14 * np.abs(oc.s) * np.abs(oc.code.astype(np.float64)).sum(1) / oc.phi
    return 1e-12 * scale


def assert_decompress_close(got, oc, rows, cols):
    ref = O.decompress(oc)
    tol = decompress_tol(oc).reshape(rows // 8, 1, cols // 8, 1)
    err = np.abs(got - ref).reshape(rows // 8, 8, cols // 8, 8)
    assert np.all((err <= tol) | (np.isnan(err) & np.isnan(ref.reshape(err.shape))))


# --- compress: bit-exact --------------------------------------------------------------------
def test_compress_plain_pair(B):
    A, Bm = W.plain_pair()
    for X in (A, Bm):
        assert_cmat_equal(B.compress(dev(X)), O.compress(X))


SHAPES = [(8, 8), (8, 1024), (1024, 8), (72, 136), (256, 264), (520, 1032)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["smooth", "noise", "wide"])
def test_compress_shapes_and_value_ranges(B, shape, kind):
    X = W.random_block_matrix(*shape, seed=sum(shape), kind=kind)
    assert_cmat_equal(B.compress(dev(X)), O.compress(X))


def test_compress_strided_and_unaligned_views(B):
    big = W.random_block_matrix(64, 200, seed=9)
    tb = dev(big)
    view = tb[:, 1:137]               # lda = 200, base 8 bytes off a 16-byte boundary
    assert view.stride(0) == 200 and view.data_ptr() % 16 == 8
    assert_cmat_equal(B.compress(view), O.compress(big[:, 1:137]))
    view2 = tb[8:40, 64:128]          # lda = 200, aligned
    assert_cmat_equal(B.compress(view2), O.compress(big[8:40, 64:128]))
    # the compressor's three load widths: 32-byte (base on 32 bytes, lda % 4
    # == 0, as view2), 16-byte (base on 16 bytes only, or lda % 4 == 2) and
    # scalar (view)
    view3 = tb[:, 2:130]              # lda = 200, base 16 bytes off a 32-byte boundary
    assert view3.data_ptr() % 32 == 16
    assert_cmat_equal(B.compress(view3), O.compress(big[:, 2:130]))
    big2 = np.concatenate([big, big[:, :2]], axis=1)
    tb2 = dev(big2)
    view4 = tb2[:, 0:136]             # lda = 202
    assert view4.stride(0) == 202 and view4.data_ptr() % 32 == 0
    assert_cmat_equal(B.compress(view4), O.compress(big2[:, 0:136]))


def special_blocks():
    rng = np.random.default_rng(77)
    blocks = [np.fromfunction(lambda i, j: (0.1 * i) * (0.1 * j), (8, 8)),   # Sec. II, Example 1
              np.full((8, 8), 2.5), np.zeros((8, 8)), -np.zeros((8, 8)),
              np.fromfunction(lambda i, j: ((i + j) % 2) * 1.0, (8, 8))]
    spike = np.zeros((8, 8)); spike[4, 3] = -7.0; blocks.append(spike)
    blocks.append(rng.standard_normal((8, 8)) * 1e-310)                     # subnormal
    blocks.append(rng.standard_normal((8, 8)) * 1e300)
    nanb = rng.standard_normal((8, 8)); nanb[2, 5] = np.nan; blocks.append(nanb)
    infb = rng.standard_normal((8, 8)); infb[0, 3] = np.inf; blocks.append(infb)
    infn = np.full((8, 8), -np.inf); blocks.append(infn)
    tiny = np.full((8, 8), 1.0); tiny[7, 7] = 1.0 + 2.0 ** -52; blocks.append(tiny)
    half = np.fromfunction(lambda i, j: np.where(i + j < 8, 0.0, 5e-324), (8, 8)); blocks.append(half)
    for _ in range(20):
        blocks.append(rng.integers(-64, 64, (8, 8)) / 32.0)
        blocks.append(np.cumsum(rng.integers(0, 9, (8, 8)), axis=1) / 16.0)   # sign-coherent
    return np.concatenate(blocks, axis=1)


def test_compress_special_values(B):
    X = special_blocks()
    assert_cmat_equal(B.compress(dev(X)), O.compress(X))


def test_compress_certification_boundaries(B, boundary_blocks):
    blk, dphi, dcode = boundary_blocks
    # the selection does reach the region where fp32 certification fails
    assert np.min(dphi) < 1e-6 and np.min(dcode) < 1e-7
    X = np.ascontiguousarray(blk.transpose(1, 0, 2).reshape(8, -1))
    assert_cmat_equal(B.compress(dev(X)), O.compress(X))
    # the same blocks with a ragged second block row and a strided view
    Y = np.concatenate([X, X[:, ::-1]], axis=0)
    tb = torch.zeros((16, Y.shape[1] + 8), dtype=torch.float64, device="cuda")
    tb[:, 8:] = dev(Y)
    assert_cmat_equal(B.compress(tb[:, 8:]), O.compress(Y))


def test_compress_uniform_block_edges(B):
    """Blocks at the edges of the compressor's integer path (one sign and one
    exponent field e, 54 <= e <= 2045, sum |N| < 2^53) and just outside it,
    bit for bit against the oracle: both signs; e = 54 and 2045 and their
    neighbours 53 and 2046; a checkerboard of 1 and 2 - 2^-52 whose integer
    slope sum reaches 2^53 (the binary64 tree then rounds); constant blocks;
    a zero entry; one entry across a binade."""
    rng = np.random.default_rng(71)
    base = 1.5 + np.cumsum(np.cumsum(rng.uniform(0, 1e-3, (8, 8)), 0), 1)      # in [1, 2)
    checker = np.where(np.add.outer(np.arange(8), np.arange(8)) % 2 == 0, 1.0, 2.0 - 2.0 ** -52)
    blocks = [base, -base, np.full((8, 8), 1.25), np.full((8, 8), -3.0), checker, -checker]
    for k in (-969, -970, 1021, 1022):          # exponent fields 54, 53, 2044, 2045 for values in [1, 2)
        blocks += [np.ldexp(base, k), -np.ldexp(base, k)]
    blocks.append(np.ldexp(base / 1.5 * 1.9, 1023 - 1))   # values in [2^1022, 2^1023]: e = 2045 and 2046
    z = base.copy(); z[3, 4] = 0.0; blocks.append(z)
    x = base.copy(); x[5, 6] = 2.0 + 1e-3; blocks.append(x)
    blocks += [np.ldexp(base, int(k)) * rng.choice([-1.0, 1.0]) for k in rng.integers(-1000, 1000, 47)]
    M = np.concatenate([np.concatenate(blocks[r * 8:(r + 1) * 8], axis=1) for r in range(len(blocks) // 8)], axis=0)
    g = B.compress(dev(M))
    assert_cmat_equal(g, O.compress(M))


def test_compress_all_blocks_sign_coherent(B):
    """Every block uniform and sign-coherent (increasing along both axes, so
    every N > 0; the negative copies all N < 0), 3 block rows of 300 blocks,
    so that every CTA of the compressor's integer pass fills all its exact-DC
    slots, whose chains reload the rows of their blocks; the last block rows
    and columns of a padded copy take the clamped reload.  Some blocks are
    constant (K = 0); with phi = 16 and K = 63 the others have their DC
    exactly on an integer code (8 | K phi).  Bit for bit against the
    oracle."""
    rng = np.random.default_rng(73)
    blocks = []
    for q in range(900):
        steps = rng.integers(1, 4, (8, 8)) * 2.0 ** -20 if q % 3 else rng.uniform(0, 1e-3, (8, 8))
        blk = 1.0 + np.cumsum(np.cumsum(steps, 0), 1)
        if q % 50 == 7:
            blk = np.full((8, 8), 1.75)
        blocks.append(-blk if q % 4 == 1 else blk)
    M = np.concatenate([np.concatenate(blocks[r * 300:(r + 1) * 300], axis=1) for r in range(3)], axis=0)
    assert_cmat_equal(B.compress(dev(M)), O.compress(M))
    R = np.ascontiguousarray(M[:21, :2395])   # edge-replicated to 24 x 2400: the blocks stay coherent
    assert_cmat_equal(B.compress_padded(dev(R)), O.compress_padded(R))


def test_compress_coherent_blocks_across_a_binade(B):
    """Sign-coherent blocks that each cross 1.0 (so none is uniform): 885 of
    900 go to the compressor's binary64 pass, whose every chunk of 128 then
    has more sign-coherent blocks than copies of D, and the dense pass forms
    the rows of the others from the input.  Bit for bit against the oracle,
    plain and with a padded copy."""
    rng = np.random.default_rng(79)
    blocks = []
    for q in range(900):
        blk = 0.99 + np.cumsum(np.cumsum(rng.uniform(0, 1e-3, (8, 8)), 0), 1)
        if q % 60 == 11:
            blk = np.full((8, 8), 1.25)
        blocks.append(-blk if q % 4 == 1 else blk)
    M = np.concatenate([np.concatenate(blocks[r * 300:(r + 1) * 300], axis=1) for r in range(3)], axis=0)
    assert_cmat_equal(B.compress(dev(M)), O.compress(M))
    R = np.ascontiguousarray(M[:23, :2397])
    assert_cmat_equal(B.compress_padded(dev(R)), O.compress_padded(R))


@pytest.mark.parametrize("shape", [(0, 0), (0, 16), (16, 0)])
def test_empty_matrices(B, shape):
    X = torch.zeros(shape, dtype=torch.float64, device="cuda")
    c = B.compress(X)
    assert c.nb == 0
    out = B.decompress(c)
    assert out.shape == shape
    assert float(B.dot(c, c).item()) == 0.0 or c.nb == 0


def test_shape_errors_are_reported(B):
    X = torch.zeros((12, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        B.compress(X)
    a = B.compress(torch.zeros((8, 16), dtype=torch.float64, device="cuda"))
    b = B.compress(torch.zeros((16, 8), dtype=torch.float64, device="cuda"))
    with pytest.raises(B.BlazError) as e:
        B.add(a, b, out=B.CMat.empty(8, 16))
    assert e.value.status == -1
    with pytest.raises(B.BlazError):
        B.dot_rowcol(a, b, 8, 0)


# --- decompress ------------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(256, 256), (72, 136), (8, 1024)])
def test_decompress_parity(B, shape):
    X = W.random_block_matrix(*shape, seed=5) if shape != (256, 256) else W.plain_pair()[0]
    oc = O.compress(X)
    got = B.decompress(B.compress(dev(X))).cpu().numpy()
    assert_decompress_close(got, oc, *shape)


def test_decompress_special_values(B):
    """NaN, infinite, subnormal and huge blocks: the finite blocks within the
    bound, the others with the oracle's NaN pattern (a NaN slope leaves M00 = f
    and makes the rest NaN)."""
    X = special_blocks()
    oc = O.compress(X)
    got = B.decompress(B.compress(dev(X))).cpu().numpy()
    ref = O.decompress(oc)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    fin = np.isfinite(ref)
    assert np.array_equal(got[~fin & ~np.isnan(ref)], ref[~fin & ~np.isnan(ref)])
    tol = np.repeat(decompress_tol(oc), 8).reshape(1, -1).repeat(8, 0)
    assert np.all(((np.abs(got - ref) <= tol) | (got == ref))[fin])


def test_decompress_into_strided_output(B):
    X = W.plain_pair()[1][:64, :96]
    oc = O.compress(X)
    out = torch.full((64, 131), 7.0, dtype=torch.float64, device="cuda")
    B.decompress(B.compress(dev(X)), out=out[:, 1:97])
    o = out.cpu().numpy()
    assert np.all(o[:, 0] == 7.0) and np.all(o[:, 97:] == 7.0)
    assert_decompress_close(o[:, 1:97], oc, 64, 96)


# --- Algorithms 1 and 2: bit-exact ---------------------------------------------------------
def test_add_sub_scale_plain_pair(B):
    A, Bm = W.plain_pair()
    ga, gb = B.compress(dev(A)), B.compress(dev(Bm))
    oa, ob = O.compress(A), O.compress(Bm)
    assert_cmat_equal(B.add(ga, gb), O.add(oa, ob))
    assert_cmat_equal(B.sub(ga, gb), O.sub(oa, ob))
    assert_cmat_equal(B.scale(ga, 3.5), O.scale(oa, 3.5))
    # repeated adds shrink phi (Eq. eq55); codes stay exact
    gs, os_ = ga, oa
    for _ in range(6):
        gs, os_ = B.add(gs, ga), O.add(os_, oa)
        assert_cmat_equal(gs, os_)


def test_scale_of_unaligned_arrays(B):
    """Arrays that start 8 bytes (f, s) or 1 byte (phi) or 4 bytes (codes) off
    a 16-byte boundary take the scalar kernel; same bits as the oracle."""
    A = W.random_block_matrix(64, 72, seed=21)
    g = B.compress(dev(A))
    nb = g.nb
    store = [torch.empty(nb + 2, dtype=torch.float64, device="cuda") for _ in range(2)] + \
            [torch.empty(nb + 16, dtype=torch.uint8, device="cuda"), torch.empty((nb + 1, 28), dtype=torch.int8, device="cuda")]
    a = B.CMat(64, 72, store[0][1:nb + 1], store[1][1:nb + 1], store[2][1:nb + 1], store[3][1:nb + 1])
    a.f.copy_(g.f), a.s.copy_(g.s), a.phi.copy_(g.phi), a.code.copy_(g.code)
    oa = O.compress(A)
    assert_cmat_equal(B.scale(a, -2.25), O.scale(oa, -2.25))
    B.scale(a, 0.75, out=a)                                 # in place
    assert_cmat_equal(a, O.scale(oa, 0.75))


@pytest.mark.parametrize("cst", [-0.97, -1.0, 2.0, 0.0, 1e-300])
def test_add_with_scaled_partner(B, cst):
    X = W.random_block_matrix(64, 64, seed=3)
    Y = np.ascontiguousarray(X.T)
    gx, gy = B.compress(dev(X)), B.compress(dev(Y))
    ox, oy = O.compress(X), O.compress(Y)
    assert_cmat_equal(B.add(gx, B.scale(gy, cst)), O.add(ox, O.scale(oy, cst)))


def test_in_place_and_aliased_outputs(B):
    A, Bm = W.plain_pair()
    ga, gb = B.compress(dev(A)), B.compress(dev(Bm))
    oa, ob = O.compress(A), O.compress(Bm)
    B.add(ga, gb, out=ga)                  # out aliases a
    assert_cmat_equal(ga, O.add(oa, ob))
    B.scale(gb, -2.25, out=gb)             # in place: only f and s rewritten
    assert_cmat_equal(gb, O.scale(ob, -2.25))


def test_add_special_values(B):
    X = special_blocks()
    Y = np.roll(X, 8, axis=1)
    gx, gy = B.compress(dev(X)), B.compress(dev(Y))
    assert_cmat_equal(B.add(gx, gy), O.add(O.compress(X), O.compress(Y)))


def test_add_tiles_ragged_aliased_and_unaligned(B):
    """The tiled kernel over 5 tiles of 256 blocks and a ragged one (25 x 41
    blocks), with out aliasing b, and the per-block kernel for code arrays
    4 bytes off a 16-byte boundary: same bits as the oracle."""
    X = W.bump_field(328, 40, rows=200)
    Y = W.bump_field(328, 41, rows=200)
    gx, gy = B.compress(dev(X)), B.compress(dev(Y))
    ox, oy = O.compress(X), O.compress(Y)
    assert_cmat_equal(B.add(gx, gy), O.add(ox, oy))
    assert_cmat_equal(B.sub(gx, gy), O.sub(ox, oy))
    s, os_ = gx, ox
    for _ in range(4):                                       # self-additions: y on integers
        s, os_ = B.add(s, gx), O.add(os_, ox)
        assert_cmat_equal(s, os_)
    gy2 = B.compress(dev(Y))
    B.sub(gx, gy2, out=gy2)                                  # out aliases b
    assert_cmat_equal(gy2, O.sub(ox, oy))
    nb = gx.nb
    store = torch.empty((nb + 1, 28), dtype=torch.int8, device="cuda")
    a = B.CMat(200, 328, gx.f, gx.s, gx.phi, store.view(-1)[4:4 + nb * 28].view(nb, 28))
    a.code.copy_(gx.code)
    assert_cmat_equal(B.add(a, gy), O.add(ox, oy))


def test_add_tiles_of_random_payloads(B):
    """The tiled kernel on payloads no compressor writes: codes over the whole
    int8 range (-128 included), slopes over 2^+-115, near-cancelling and equal
    slopes (huge and integer-valued beta, saturated codes, tiles with more
    listed blocks than the list holds), zero slopes; 7 tiles and a ragged
    one.  Same bits as the oracle for the sum and the difference."""
    rng = np.random.default_rng(77)
    n = 7 * 256 + 37
    mats = []
    for _ in range(2):
        m = O.CMat.empty(8, 8 * n)
        m.f[:] = rng.normal(size=n)
        m.s[:] = rng.choice([-1.0, 1.0], n) * np.exp(rng.uniform(-80, 80, n))
        m.phi[:] = rng.integers(1, 256, n)
        m.code[:] = rng.integers(-128, 128, (n, 28))
        mats.append(m)
    a, b = mats
    b.s[: n // 8] = -a.s[: n // 8] * (1 + rng.uniform(-1e-12, 1e-12, n // 8))
    b.s[n // 8: n // 4] = a.s[n // 8: n // 4]
    b.s[n // 4: n // 4 + 64] = 0.0
    a.s[n // 4 + 64: n // 4 + 80] = 0.0
    b.phi[n // 2: n // 2 + 300] = a.phi[n // 2: n // 2 + 300]
    b.code[n // 2: n // 2 + 300] = a.code[n // 2: n // 2 + 300]

    def gpu(m):
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        return B.CMat(m.rows, m.cols, t(m.f), t(m.s), t(m.phi), t(m.code))

    ga, gb = gpu(a), gpu(b)
    assert_cmat_equal(B.add(ga, gb), O.add(a, b))
    assert_cmat_equal(B.sub(ga, gb), O.sub(a, b))
    assert_cmat_equal(B.add(gb, ga), O.add(b, a))


# --- dot products and matmul -----------------------------------------------------------------
def test_dot_plain_pair(B):
    A, Bm = W.plain_pair()
    ga, gb = B.compress(dev(A)), B.compress(dev(Bm))
    v = float(B.dot(ga, gb).item())
    ref, absref = O.dot(O.compress(A), O.compress(Bm))
    assert abs(v - ref) <= 1e-12 * absref
    # deterministic: same bits again
    assert float(B.dot(ga, gb).item()) == v


@pytest.mark.parametrize("shape", [(8, 8), (200, 328), (1032, 1000), (64, 8 * 129)])
def test_dot_ragged_tiles_and_extreme_codes(B, shape):
    """The tensor-core dot over tiles of 128 blocks: one block, a ragged last
    tile, several tiles per CTA; then codes of +-127 everywhere (the largest
    slice products) and mixed-sign slopes."""
    r, c = shape
    X = W.random_block_matrix(r, c, seed=r + c)
    Y = W.random_block_matrix(r, c, seed=r + c + 1, kind="noise")
    gx, gy = B.compress(dev(X)), B.compress(dev(Y))
    ox, oy = O.compress(X), O.compress(Y)
    v = float(B.dot(gx, gy).item())
    ref, absref = O.dot(ox, oy)
    assert abs(v - ref) <= 1e-12 * absref
    rng = np.random.default_rng(r)
    for m, om in ((gx, ox), (gy, oy)):
        codes = rng.choice(np.array([-127, 127], np.int8), size=om.code.shape)
        om.code[:] = codes
        om.s[:] = om.s * rng.choice([-1.0, 1.0], size=om.s.shape)
        m.code.copy_(torch.from_numpy(om.code))
        m.s.copy_(torch.from_numpy(om.s))
    v = float(B.dot(gx, gy).item())
    ref, absref = O.dot(ox, oy)
    assert abs(v - ref) <= 1e-12 * absref


@pytest.mark.parametrize("ij", [(17, 200), (0, 0), (255, 255), (100, 3)])
def test_dot_rowcol_plain_pair(B, ij):
    A, Bm = W.plain_pair()
    ga, gb = B.compress(dev(A)), B.compress(dev(Bm))
    v = float(B.dot_rowcol(ga, gb, *ij).item())
    ref, absref = O.dot_rowcol(O.compress(A), O.compress(Bm), *ij)
    assert abs(v - ref) <= 1e-12 * absref


@pytest.mark.parametrize("ij", [(17, 30), (0, 0), (135, 71), (64, 8), (7, 63)])
def test_dot_rowcol_rectangular(B, ij):
    """Algorithm 3 for a general n x k times k x m pair (Sec. III): A is
    136 x 1032 (129 block columns), B is 1032 x 72 (9 block columns), so a
    kernel that indexed one operand with the other's block-column count
    reads the wrong blocks."""
    A = W.random_block_matrix(136, 1032, seed=41)
    Bm = W.random_block_matrix(1032, 72, seed=42)
    ga, gb = B.compress(dev(A)), B.compress(dev(Bm))
    v = float(B.dot_rowcol(ga, gb, *ij).item())
    ref, absref = O.dot_rowcol(O.compress(A), O.compress(Bm), *ij)
    assert abs(v - ref) <= 1e-12 * absref


def test_dot_rowcol_grid_stride(B):
    """k = 40000 (5000 k-blocks): more k-blocks than one wave of 16-lane teams
    over the SMs (16 x 152 = 2432 on a GB300), so every team loops."""
    A = W.random_block_matrix(16, 40000, seed=43)
    Bm = W.random_block_matrix(40000, 24, seed=44)
    ga, gb = B.compress(dev(A)), B.compress(dev(Bm))
    oa, ob = O.compress(A), O.compress(Bm)
    for ij in [(3, 17), (15, 0), (8, 23)]:
        v = float(B.dot_rowcol(ga, gb, *ij).item())
        ref, absref = O.dot_rowcol(oa, ob, *ij)
        assert abs(v - ref) <= 1e-12 * absref


def test_dot_rowcol_bandwidth_sweep_launch(B):
    """The benchmark's own call: line 17 times column 200 of two 16384^2 bump
    fields.  The oracle compresses only the block row of A and the block
    column of B the line and the column live in (compression is block-local,
    so these are the same blocks)."""
    n = 16384
    ta = W.bump_field_torch(n, n, "cuda")
    tb = W.bump_field_torch(n, n + 1, "cuda")
    ga, gb = B.compress(ta), B.compress(tb)
    v = float(B.dot_rowcol(ga, gb, 17, 200).item())
    oa = O.compress(ta[16:24].cpu().numpy())
    ob = O.compress(tb[:, 200:208].contiguous().cpu().numpy())
    ref, absref = O.dot_rowcol(oa, ob, 1, 0)
    assert abs(v - ref) <= 1e-12 * absref
    del ta, tb, ga, gb
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n,k,m", [(256, 256, 256), (72, 136, 50), (8, 8, 1), (64, 1024, 129)])
def test_matmul_fp64(B, n, k, m):
    A = W.random_block_matrix(n, k, seed=n + k)
    Bd = W.smoothed_normal(k, m, seed=7)
    ga = B.compress(dev(A))
    C = B.matmul(ga, dev(Bd), mode="fp64").cpu().numpy()
    oa = O.compress(A)
    ref = O.matmul(oa, Bd)
    bound = np.abs(O.decompress(oa)) @ np.abs(Bd)
    assert np.all(np.abs(C - ref) <= 1e-12 * bound + 1e-300)


# --- full sizes of the bandwidth sweep (launch configuration of the benchmark) ---------------
def _sample_blocks(nbr, nbc, rng, count=3000):
    idx = set(rng.integers(0, nbr * nbc, count).tolist())
    idx |= set(range(min(nbc, 64)))                        # first block-row head
    idx |= set(range(nbr * nbc - min(nbc, 64), nbr * nbc))  # last block-row tail
    idx |= {b * nbc for b in range(0, nbr, max(1, nbr // 64))}
    return np.array(sorted(idx), dtype=np.int64)


def _gather_blocks(t, idx, nbc):
    """Stack the listed 8x8 blocks of a device matrix vertically, on the host."""
    bi = torch.from_numpy(idx // nbc).cuda()
    bj = torch.from_numpy(idx % nbc).cuda()
    r = (bi[:, None] * 8 + torch.arange(8, device="cuda")[None, :])          # [n, 8]
    c = (bj[:, None] * 8 + torch.arange(8, device="cuda")[None, :])          # [n, 8]
    blk = t[r[:, :, None], c[:, None, :]]                                      # [n, 8, 8]
    return blk.reshape(-1, 8).cpu().numpy()


@pytest.mark.parametrize("n", [1024, 4096, 16384])
def test_bandwidth_sweep_full_size_sampled(B, n):
    ta = W.bump_field_torch(n, n, "cuda")
    tb = W.bump_field_torch(n, n + 1, "cuda")
    ga, gb = B.compress(ta), B.compress(tb)
    nbc = n // 8
    idx = _sample_blocks(nbc, nbc, np.random.default_rng(n))
    oa = O.compress(_gather_blocks(ta, idx, nbc))     # oracle compresses the same blocks
    ob = O.compress(_gather_blocks(tb, idx, nbc))
    assert_cmat_equal(ga, oa, idx)
    assert_cmat_equal(gb, ob, idx)
    gs = B.add(ga, gb)
    assert_cmat_equal(gs, O.add(oa, ob), idx)
    gc = B.scale(ga, 3.5)
    assert_cmat_equal(gc, O.scale(oa, 3.5), idx)
    dec = B.decompress(ga)
    got = _gather_blocks(dec, idx, nbc)
    assert_decompress_close(got, oa, got.shape[0], 8)
    del dec, ta, tb
    torch.cuda.empty_cache()


def _oracle_dot_chunked(A, Bm, nchunks):
    """Oracle dot of the oracle's own compressions, evaluated over disjoint
    block-row chunks in parallel threads and summed exactly (math.fsum)."""
    O.dct_tables()                        # initialise the oracle's tables before threading
    rows = A.shape[0]
    step = max(8, (rows // nchunks) // 8 * 8)
    spans = [(r, min(rows, r + step)) for r in range(0, rows, step)]

    def one(sp):
        a = O.compress(A[sp[0]:sp[1]])
        b = O.compress(Bm[sp[0]:sp[1]])
        return O.dot(a, b)

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        parts = list(ex.map(one, spans))
    return math.fsum(p[0] for p in parts), math.fsum(p[1] for p in parts)


@pytest.mark.parametrize("n", [1024, 4096])
def test_bandwidth_sweep_dot_full_size(B, n):
    A = W.bump_field(n, n)
    Bm = W.bump_field(n, n + 1)
    v = float(B.dot(B.compress(dev(A)), B.compress(dev(Bm))).item())
    ref, absref = _oracle_dot_chunked(A, Bm, 16)
    assert abs(v - ref) <= 1e-12 * absref


def test_precision_config_matmul_fp64_sampled(B):
    n = 4096
    ta = W.bump_field_torch(n, n, "cuda")
    Bd = W.smoothed_normal(n, n, seed=7)
    ga = B.compress(ta)
    C = B.matmul(ga, dev(Bd), mode="fp64")
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(n, 12, replace=False))
    # the oracle compresses the rows' block-rows itself
    blockrows = sorted({r // 8 for r in rows})
    for br in blockrows:
        Arow = ta[br * 8:(br + 1) * 8].cpu().numpy()
        oa = O.compress(Arow)
        jj = rng.choice(n, 64, replace=False)
        ii = np.repeat(np.array([r - br * 8 for r in rows if r // 8 == br]), len(jj))
        jj = np.tile(jj, len(ii) // len(jj))
        ref, bound = O.matmul_entries(oa, Bd, ii, jj)
        got = C[torch.from_numpy(ii + br * 8).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * bound)


# --- split-precision tensor-core product -----------------------------------------------------
@pytest.mark.parametrize("n,k,m", [(256, 256, 256), (72, 136, 50), (8, 8, 1), (64, 8, 64), (64, 1024, 129),
                                   (384, 64, 520)])
def test_matmul_split_bf16(B, n, k, m):
    A = W.random_block_matrix(n, k, seed=n + k)
    Bd = W.smoothed_normal(k, m, seed=7)
    ga = B.compress(dev(A))
    C = B.matmul(ga, dev(Bd), mode="split_bf16").cpu().numpy()
    assert B.device_status() == 0
    oa = O.compress(A)
    ref = O.matmul(oa, Bd)
    bound = np.abs(O.decompress(oa)) @ np.abs(Bd)
    err = np.abs(C - ref)
    assert np.all(err <= split_bf16_tol(k) * bound + 1e-300), np.max(err / (bound + 1e-300))
    if k >= 1024:
        assert np.all(err <= SPLIT_BF16_LARGE_K_TOL * bound + 1e-300), np.max(err / (bound + 1e-300))


def test_matmul_split_bf16_empty_inner_dimension(B):
    ga = B.compress(torch.zeros((16, 0), dtype=torch.float64, device="cuda"))
    C = B.matmul(ga, torch.zeros((0, 24), dtype=torch.float64, device="cuda"), mode="split_bf16")
    assert C.shape == (16, 24) and float(C.abs().max()) == 0.0


@pytest.mark.parametrize("mode", ["fp64", "split_bf16"])
@pytest.mark.parametrize("n,k,m", [(8, 8, 8), (72, 136, 64), (264, 256, 520)])
def test_matmul_compressed_by_compressed(B, mode, n, k, m):
    """A_hat @ B_hat (both compressed) against the oracle's product of the two
    decompressions, with the tolerance of the matching dense-B mode."""
    A = W.random_block_matrix(n, k, seed=n + k)
    Bm = W.random_block_matrix(k, m, seed=k + m + 1)
    ga, gb = B.compress(dev(A)), B.compress(dev(Bm))
    C = B.matmul_cc(ga, gb, mode=mode).cpu().numpy()
    assert B.device_status() == 0
    oa, ob = O.compress(A), O.compress(Bm)
    ref = O.matmul_cc(oa, ob)
    bound = np.abs(O.decompress(oa)) @ np.abs(O.decompress(ob))
    tol = 1e-12 if mode == "fp64" else split_bf16_tol(k)
    err = np.abs(C - ref)
    assert np.all(err <= tol * bound + 1e-300), np.max(err / (bound + 1e-300))


def test_matmul_compressed_by_compressed_edges(B):
    import ctypes

    a = B.compress(dev(W.random_block_matrix(16, 24, seed=3)))
    b = B.compress(dev(W.random_block_matrix(16, 8, seed=4)))
    out = torch.zeros((16, 8), dtype=torch.float64, device="cuda")
    da, db = a.desc(), b.desc()
    rc = B.lib().blaz_matmul_cc(ctypes.byref(da), ctypes.byref(db), out.data_ptr(), 8, 0,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1                                       # inner dimensions differ: BLAZ_ERR_SHAPE
    e0 = B.compress(torch.zeros((16, 0), dtype=torch.float64, device="cuda"))
    e1 = B.compress(torch.zeros((0, 24), dtype=torch.float64, device="cuda"))
    C = B.matmul_cc(e0, e1)
    assert C.shape == (16, 24) and float(C.abs().max()) == 0.0
    # output into a strided view (ldc > m)
    A = W.random_block_matrix(40, 32, seed=5)
    Bm = W.random_block_matrix(32, 48, seed=6)
    big = torch.full((40, 72), 7.0, dtype=torch.float64, device="cuda")
    B.matmul_cc(B.compress(dev(A)), B.compress(dev(Bm)), out=big[:, 8:56])
    oa, ob = O.compress(A), O.compress(Bm)
    ref = O.matmul_cc(oa, ob)
    bound = np.abs(O.decompress(oa)) @ np.abs(O.decompress(ob))
    got = big.cpu().numpy()
    assert np.all(np.abs(got[:, 8:56] - ref) <= 1e-12 * bound + 1e-300)
    assert np.all(got[:, :8] == 7.0) and np.all(got[:, 56:] == 7.0)


@pytest.mark.parametrize("mode", ["fp64", "split_bf16"])
def test_precision_config_max_relative_error(B, mode, record_property):
    """Precision workload: compressed 4096^2 bump field times a smoothed N(0,1)
    4096^2 matrix; sampled entries against the oracle (which compresses the
    sampled block-rows itself).  Reports the max relative errors."""
    n = 4096
    ta = W.bump_field_torch(n, n, "cuda")
    Bd = W.smoothed_normal(n, n, seed=7)
    ga = B.compress(ta)
    C = B.matmul(ga, dev(Bd), mode=mode)
    assert B.device_status() == 0
    rng = np.random.default_rng(2)
    worst_comp = worst_rel = 0.0
    for br in sorted(rng.choice(n // 8, 6, replace=False)):
        oa = O.compress(ta[br * 8:(br + 1) * 8].cpu().numpy())
        ii = np.repeat(np.arange(8), 48)
        jj = np.tile(rng.choice(n, 48, replace=False), 8)
        ref, bound = O.matmul_entries(oa, Bd, ii, jj)
        got = C[torch.from_numpy(ii + br * 8).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
        comp = np.abs(got - ref) / bound
        worst_comp = max(worst_comp, float(comp.max()))
        big = np.abs(ref) > 1e-8 * np.abs(ref).max()
        worst_rel = max(worst_rel, float((np.abs(got - ref)[big] / np.abs(ref[big])).max()))
    tol = 1e-12 if mode == "fp64" else split_bf16_tol(n)
    print(f"\n[{mode}] max componentwise error {worst_comp:.3e}, max relative error {worst_rel:.3e}")
    record_property("max_componentwise_error", worst_comp)
    record_property("max_relative_error", worst_rel)
    assert worst_comp <= tol
    if mode == "split_bf16":
        assert worst_comp <= SPLIT_BF16_LARGE_K_TOL


# --- the stages of one block (Examples 1-5 of Sec. II) ------------------------------------------
def _stage_blocks():
    from conftest import load_golden

    g = load_golden("example_xy.txt")
    ex = np.array([[float(x) for x in row] for row in g["A"]])
    rng = np.random.default_rng(77)
    blocks = [ex, np.full((8, 8), 3.25), W.random_block_matrix(8, 8, 4), W.random_block_matrix(8, 8, 5, "noise"),
              W.random_block_matrix(8, 8, 6, "wide"), np.cumsum(np.cumsum(rng.random((8, 8)), 0), 1)]
    return blocks


@pytest.mark.parametrize("k", range(6))
def test_debug_block_stages_match_the_oracle(B, k):
    """Every stage (delta, K, the slope sum, s, dprime, s_max, the prediction
    indexes, all 64 DCT coefficients, m, phi, f, codes) bit for bit against
    the oracle, on the paper's worked example, a constant block and random
    smooth, rough and wide-range blocks."""
    M = _stage_blocks()[k]
    g = B.debug_block_stages(dev(M.reshape(64)))
    o = O.block_stages(M)
    for key in ("delta", "dprime", "dct"):
        same_bits(g[key].reshape(-1), o[key].reshape(-1))
    for key in ("sum_abs", "s", "s_max", "m", "f"):
        same_bits([g[key]], [o[key]])
    assert g["K"] == o["K"] and g["phi"] == o["phi"]
    assert np.array_equal(g["psi"], o["psi"])
    assert np.array_equal(g["code"], o["code"])
    # the stored block equals the compressor's
    c = B.compress(dev(M)).to_host()
    assert c[2][0] == g["phi"] and np.array_equal(c[3][0], g["code"])
    same_bits(c[1][:1], [g["s"]])
