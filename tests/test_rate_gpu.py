"""GPU parity of the tunable-rate entry points (the first r DCT rows and
columns kept, r = 1..8) against the oracle: codes, phi, f and s of compress,
add, sub and scale bit for bit; decompression within
1e-12 (|f| + 14 |s| sum|c| / phi) per block, the bound of the 28-code path
(the recurrence adds at most 14 inverse-DCT terms of size <= |s| sum|c|/phi)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

RATES = list(range(1, 9))


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


def assert_same(g, o):
    f, s, phi, code = g.to_host()
    assert np.array_equal(phi, o.phi)
    assert np.array_equal(code, o.code)
    same_bits(f, o.f)
    same_bits(s, o.s)


def mixed_matrix(seed=3):
    """72 x 136 (153 blocks: a ragged last CTA): smooth, rough and
    wide-range rows plus special blocks (constant, zero, NaN, infinities,
    subnormal, Sec. II's Example 1)."""
    rng = np.random.default_rng(seed)
    X = np.concatenate([W.random_block_matrix(24, 136, seed=seed + k, kind=kind)
                        for k, kind in enumerate(["smooth", "noise", "wide"])], axis=0)
    X[0:8, 0:8] = np.fromfunction(lambda i, j: (0.1 * i) * (0.1 * j), (8, 8))
    X[0:8, 8:16] = 2.5
    X[0:8, 16:24] = 0.0
    X[8:16, 8:16] = rng.standard_normal((8, 8)) * 1e-310
    X[8, 20] = np.nan
    X[16, 30] = np.inf
    X[16:24, 40:48] = -np.inf
    X[24:32, 48:56] = rng.standard_normal((8, 8)) * 1e300
    return X


@pytest.mark.parametrize("r", RATES)
def test_compress_rate_bit_exact(B, r):
    X = mixed_matrix()
    assert_same(B.compress_rate(dev(X), r), O.compress_rate(X, r))


def test_rate_two_matches_the_28_code_kernels(B):
    A, Bm = W.plain_pair()
    a2, a = B.compress_rate(dev(A), 2), B.compress(dev(A))
    for x, y in zip(a2.to_host(), a.to_host()):
        assert np.array_equal(np.asarray(x).view(np.uint8), np.asarray(y).view(np.uint8))


@pytest.mark.parametrize("r", RATES)
def test_decompress_rate(B, r):
    X = mixed_matrix(5)
    oc = O.compress_rate(X, r)
    got = B.decompress_rate(B.compress_rate(dev(X), r)).cpu().numpy()
    ref = O.decompress_rate(oc, r)
    scale = np.abs(oc.f) + 14 * np.abs(oc.s) * np.abs(oc.code.astype(np.float64)).sum(1) / oc.phi
    tol = (1e-12 * scale).reshape(oc.rows // 8, 1, oc.cols // 8, 1)
    err = np.abs(got - ref).reshape(oc.rows // 8, 8, oc.cols // 8, 8)
    # blocks with a NaN slope (NaN or infinite inputs) are NaN past M00 on both sides
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    ok = (err <= tol) | np.isnan(ref.reshape(err.shape)) | (got == ref).reshape(err.shape)
    assert np.all(ok), np.argwhere(~ok)[:5]


@pytest.mark.parametrize("r", RATES)
def test_add_sub_scale_rate_bit_exact(B, r):
    X, Y = mixed_matrix(7), mixed_matrix(11)[:, ::-1]
    ga, gb = B.compress_rate(dev(X), r), B.compress_rate(dev(Y), r)
    oa, ob = O.compress_rate(X, r), O.compress_rate(Y, r)
    assert_same(B.add_rate(ga, gb), O.add_rate(oa, ob, r))
    assert_same(B.sub_rate(ga, gb), O.add_rate(oa, ob, r, sub=True))
    for c in (-0.97, 3.5, 0.0):
        assert_same(B.scale_rate(ga, c), O.scale_rate(oa, c))


@pytest.mark.parametrize("r", [1, 3, 8])
def test_rate_ops_in_place_and_aliased(B, r):
    X, Y = mixed_matrix(2), mixed_matrix(4)
    oa, ob = O.compress_rate(X, r), O.compress_rate(Y, r)
    ga, gb = B.compress_rate(dev(X), r), B.compress_rate(dev(Y), r)
    B.add_rate(ga, gb, out=ga)                     # out aliases a
    want = O.add_rate(oa, ob, r)
    assert_same(ga, want)
    B.sub_rate(gb, ga, out=ga)                     # out aliases b
    want = O.add_rate(ob, want, r, sub=True)
    assert_same(ga, want)
    B.scale_rate(ga, -2.0, out=ga)                 # in place
    assert_same(ga, O.scale_rate(want, -2.0))


@pytest.mark.parametrize("r", [1, 4])
def test_rate_strided_view_and_large_sampled(B, r):
    big = W.random_block_matrix(64, 200, seed=9)
    tb = dev(big)
    view = tb[:, 1:137]                            # lda = 200, base not 16-byte aligned
    assert_same(B.compress_rate(view, r), O.compress_rate(big[:, 1:137], r))
    # 2048 x 2048 (65536 blocks, a full grid of CTAs): sampled blocks
    n = 2048
    A = W.bump_field(n, seed=21)
    g = B.compress_rate(dev(A), r)
    f, s, phi, code = g.to_host()
    rng = np.random.default_rng(1)
    nbc = n // 8
    idx = np.unique(np.concatenate([rng.integers(0, nbc * nbc, 200), [0, nbc - 1, nbc * nbc - 1]]))
    sub = np.concatenate([A[8 * (b // nbc):8 * (b // nbc) + 8, 8 * (b % nbc):8 * (b % nbc) + 8] for b in idx],
                         axis=1)
    oc = O.compress_rate(sub, r)
    assert np.array_equal(phi[idx], oc.phi) and np.array_equal(code[idx], oc.code)
    same_bits(f[idx], oc.f)
    same_bits(s[idx], oc.s)


def test_rate_argument_errors(B):
    X = dev(mixed_matrix())
    for r in (0, 9, -3):
        with pytest.raises(ValueError):
            B.keep_count(r)
    a = B.compress_rate(X, 3)
    b = B.compress_rate(X, 5)
    with pytest.raises(ValueError):
        B.add_rate(a, b)
    d = a.desc()
    assert B.lib().blaz_compress_rate(X.data_ptr(), 136, 9, d, None) == -9
    assert B.lib().blaz_decompress_rate(d, 0, X.data_ptr(), 136, None) == -9
    e = B.CMat.empty(0, 16, rate=4)
    assert B.decompress_rate(e).shape == (0, 16)


@pytest.mark.parametrize("r", [1, 4, 8])
def test_compress_rate_certification_boundaries(B, r, boundary_blocks):
    """Blocks whose phi or codes sit closest to a truncation boundary: the
    fp32 decisions must defer them to the exact fix-up."""
    blk, _, _ = boundary_blocks
    X = np.ascontiguousarray(blk.transpose(1, 0, 2).reshape(8, -1))
    assert_same(B.compress_rate(dev(X), r), O.compress_rate(X, r))


@pytest.mark.parametrize("r", [2, 5, 8])
def test_add_rate_structural_ties(B, r):
    """A + A and A - A (equal phi and codes put beta_1 c_1 +- beta_2 c_2 on an
    integer: the binary64 pass decides them) and smooth + rough pairs."""
    X = W.bump_field(256, seed=3)
    Y = W.random_block_matrix(256, 256, seed=8, kind="noise")
    ga, gb = B.compress_rate(dev(X), r), B.compress_rate(dev(Y), r)
    oa, ob = O.compress_rate(X, r), O.compress_rate(Y, r)
    assert_same(B.add_rate(ga, ga), O.add_rate(oa, oa, r))
    assert_same(B.sub_rate(ga, ga), O.add_rate(oa, oa, r, sub=True))
    assert_same(B.add_rate(ga, gb), O.add_rate(oa, ob, r))
    assert_same(B.sub_rate(gb, ga), O.add_rate(ob, oa, r, sub=True))


@pytest.mark.parametrize("r", RATES)
@pytest.mark.parametrize("shape", [(8, 8), (72, 136), (264, 1000)])
def test_dot_rate(B, r, shape):
    """Flattened dot within 1e-12 sum |A_hat B_hat|: one block, a ragged last
    group of 16 blocks, many groups per CTA; deterministic."""
    X = W.random_block_matrix(*shape, seed=shape[0] + r)
    Y = W.random_block_matrix(*shape, seed=shape[1] + r, kind="noise")
    gx, gy = B.compress_rate(dev(X), r), B.compress_rate(dev(Y), r)
    ref, absref = O.dot_rate(O.compress_rate(X, r), O.compress_rate(Y, r), r)
    v = float(B.dot_rate(gx, gy).item())
    assert abs(v - ref) <= 1e-12 * absref
    assert float(B.dot_rate(gx, gy).item()) == v


@pytest.mark.parametrize("r", [1, 4, 8])
def test_dot_rate_extreme_codes(B, r):
    """Codes of +-127 everywhere (the largest slice products) and slopes of
    both signs."""
    X = W.random_block_matrix(64, 8 * 129, seed=5)
    ox, oy = O.compress_rate(X, r), O.compress_rate(X[:, ::-1].copy(), r)
    rng = np.random.default_rng(r)
    for om in (ox, oy):
        om.code[:] = rng.choice(np.array([-127, 127], np.int8), size=om.code.shape)
        om.s[:] = om.s * rng.choice([-1.0, 1.0], size=om.s.shape)
    gx, gy = B.CMat.empty(64, 8 * 129, rate=r), B.CMat.empty(64, 8 * 129, rate=r)
    for g, om in ((gx, ox), (gy, oy)):
        g.f.copy_(torch.from_numpy(om.f))
        g.s.copy_(torch.from_numpy(om.s))
        g.phi.copy_(torch.from_numpy(om.phi))
        g.code.copy_(torch.from_numpy(om.code))
    ref, absref = O.dot_rate(ox, oy, r)
    assert abs(float(B.dot_rate(gx, gy).item()) - ref) <= 1e-12 * absref


@pytest.mark.parametrize("r", [1, 2, 5, 8])
@pytest.mark.parametrize("ij", [(17, 200), (0, 0), (255, 255), (100, 3)])
def test_dot_rowcol_rate(B, r, ij):
    A, Bm = W.plain_pair()
    ga, gb = B.compress_rate(dev(A), r), B.compress_rate(dev(Bm), r)
    ref, absref = O.dot_rowcol_rate(O.compress_rate(A, r), O.compress_rate(Bm, r), r, *ij)
    assert abs(float(B.dot_rowcol_rate(ga, gb, *ij).item()) - ref) <= 1e-12 * absref


@pytest.mark.parametrize("r", [1, 3, 8])
def test_dot_rowcol_rate_rectangular_and_grid_stride(B, r):
    """Algorithm 3 at rate r for general shapes: A 136 x 1032 (129 block
    columns) times B 1032 x 72 (9 block columns), then k = 40000 (5000
    k-blocks, more than one wave of 16-lane teams, so every team loops)."""
    for (n, k, m), seeds, ijs in [((136, 1032, 72), (51, 52), [(17, 30), (135, 71), (7, 63)]),
                                   ((16, 40000, 24), (53, 54), [(3, 17), (15, 0)])]:
        A = W.random_block_matrix(n, k, seed=seeds[0])
        Bm = W.random_block_matrix(k, m, seed=seeds[1])
        ga, gb = B.compress_rate(dev(A), r), B.compress_rate(dev(Bm), r)
        oa, ob = O.compress_rate(A, r), O.compress_rate(Bm, r)
        for ij in ijs:
            ref, absref = O.dot_rowcol_rate(oa, ob, r, *ij)
            assert abs(float(B.dot_rowcol_rate(ga, gb, *ij).item()) - ref) <= 1e-12 * absref


@pytest.mark.parametrize("r", [1, 3, 8])
@pytest.mark.parametrize("n,k,m", [(72, 136, 50), (256, 256, 256)])
def test_matmul_rate(B, r, n, k, m):
    from conftest import split_bf16_tol

    A = W.random_block_matrix(n, k, seed=n + k)
    Bd = W.smoothed_normal(k, m, seed=7)
    ga = B.compress_rate(dev(A), r)
    ref, absref = O.matmul_rate(O.compress_rate(A, r), r, Bd)
    got = B.matmul_rate(ga, dev(Bd)).cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-12 * absref)
    got = B.matmul_rate(ga, dev(Bd), mode="split_bf16").cpu().numpy()
    assert np.all(np.abs(got - ref) <= split_bf16_tol(k) * absref)
    # compressed x compressed at the same rate
    Y = W.random_block_matrix(k, m + (-m % 8), seed=k)
    gy = B.compress_rate(dev(Y), r)
    ref2, abs2 = O.matmul_rate(O.compress_rate(A, r), r, O.decompress_rate(O.compress_rate(Y, r), r))
    got2 = B.matmul_cc_rate(ga, gy).cpu().numpy()
    assert np.all(np.abs(got2 - ref2) <= 1e-12 * abs2)


@pytest.mark.parametrize("r", [2, 8])
def test_rate_ops_at_the_timed_size_sampled(B, r):
    """4096 x 4096 bump fields (the size bench.py times the rate kernels at):
    codes, phi, f and s of compress and add on 256 sampled blocks against the
    oracle, decompression of those blocks within the bound, and the flattened
    dot against the oracle's exact sum."""
    n = 4096
    X, Y = W.bump_field(n, seed=n), W.bump_field(n, seed=n + 1)
    gx, gy = B.compress_rate(dev(X), r), B.compress_rate(dev(Y), r)
    gs = B.add_rate(gx, gy)
    back = B.decompress_rate(gx).cpu().numpy()
    nbc = n // 8
    rng = np.random.default_rng(r)
    idx = np.unique(np.concatenate([rng.integers(0, nbc * nbc, 256), [0, nbc - 1, nbc * nbc - 1]]))

    def blocks(M):
        return np.concatenate([M[8 * (b // nbc):8 * (b // nbc) + 8, 8 * (b % nbc):8 * (b % nbc) + 8] for b in idx],
                              axis=1)

    ox, oy = O.compress_rate(blocks(X), r), O.compress_rate(blocks(Y), r)
    for g, o in ((gx, ox), (gs, O.add_rate(ox, oy, r))):
        f, s, phi, code = g.to_host()
        assert np.array_equal(phi[idx], o.phi) and np.array_equal(code[idx], o.code)
        same_bits(f[idx], o.f)
        same_bits(s[idx], o.s)
    ref = O.decompress_rate(ox, r)
    scale = np.abs(ox.f) + 14 * np.abs(ox.s) * np.abs(ox.code.astype(np.float64)).sum(1) / ox.phi
    err = np.abs(blocks(back) - ref).reshape(8, len(idx), 8).max(axis=(0, 2))
    assert np.all(err <= 1e-12 * scale)
    # the whole-field dot against the oracle's (every block)
    v = float(B.dot_rate(gx, gy).item())
    ref_v, abs_v = O.dot_rate(O.compress_rate(X, r), O.compress_rate(Y, r), r)
    assert abs(v - ref_v) <= 1e-12 * abs_v


def test_worked_example_on_the_gpu_at_every_rate(B):
    """Sec. II, Example 5's printed P' (all 64 entries) in each rate's order,
    computed by the GPU compressor."""
    from conftest import load_golden

    g = load_golden("example_xy.txt")
    P1 = np.array([[int(x) for x in row] for row in g["P'"]])
    A = np.fromfunction(lambda i, j: (0.1 * i) * (0.1 * j), (8, 8))
    for r in RATES:
        f, s, phi, code = B.compress_rate(dev(A), r).to_host()
        rows = [(i, j) for i in range(r) for j in range(8)] + [(i, j) for i in range(r, 8) for j in range(r)]
        assert list(code[0]) == [P1[i, j] for i, j in rows], r
        assert phi[0] == int(g["phi"][0][0])


@pytest.mark.parametrize("r", [1, 5, 8])
def test_decompress_rate_into_strided_views(B, r):
    """Output rows longer than the matrix (lda = cols + 8) and a base 8 bytes
    off a 16-byte boundary (no vector stores): same values as the contiguous
    decompression, the entries outside the view untouched."""
    X = W.random_block_matrix(72, 136, seed=r)
    g = B.compress_rate(dev(X), r)
    want = B.decompress_rate(g).cpu().numpy()
    for off in (0, 1):
        big = torch.full((72, 136 + 8 + off), -7.0, dtype=torch.float64, device="cuda")
        view = big[:, off:off + 136]
        B.decompress_rate(g, out=view)
        got = big.cpu().numpy()
        assert np.array_equal(got[:, off:off + 136], want)
        assert np.all(got[:, :off] == -7.0) and np.all(got[:, off + 136:] == -7.0)
