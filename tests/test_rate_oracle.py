"""Pins of the oracle's tunable-rate functions (Sec. VI names a tunable
compression rate as future work; the reading here keeps the first r rows and
the first r columns of each block's DCT, r = 1..8).

What fixes them besides the oracle itself:
* r = 2 is the paper's 28-code format, whose oracle is pinned to the worked
  example of Sec. II: compress, decompress, add and sub must agree bit for bit;
* the kept set and its order follow from the reading alone (counted here by
  brute force over the 8x8 grid); at r = 8 every code is trunc(X phi) of the
  block's full DCT from the pinned stage-by-stage oracle, row-major;
* quantization is the only loss at r = 8, so the round trip obeys a bound
  derived from the orthonormality of the DCT and the recurrence of the
  inverse normalization (see test_full_rate_round_trip_bound);
* keeping more coefficients on a smooth field lowers the error."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def kept_set(r):
    """Kept (i, j) at rate r in storage order: rows 0..r-1, then the first r
    columns of the remaining rows."""
    rows = [(i, j) for i in range(r) for j in range(8)]
    cols = [(i, j) for i in range(r, 8) for j in range(r)]
    return rows + cols


def test_keep_counts_match_the_kept_set():
    for r in range(1, 9):
        brute = sum(1 for i in range(8) for j in range(8) if i < r or j < r)
        assert O.keep_count(r) == brute == len(kept_set(r))
    assert [O.keep_count(r) for r in range(1, 9)] == [15, 28, 39, 48, 55, 60, 63, 64]
    for r in (0, 9, -1):
        with pytest.raises(Exception):
            O.keep_count(r)


def test_rate_two_is_the_paper_format():
    A, B = W.plain_pair()
    a2, b2 = O.compress_rate(A, 2), O.compress_rate(B, 2)
    a, b = O.compress(A), O.compress(B)
    for x, y in ((a2, a), (b2, b)):
        assert np.array_equal(x.f, y.f) and np.array_equal(x.s, y.s)
        assert np.array_equal(x.phi, y.phi) and np.array_equal(x.code, y.code)
    assert np.array_equal(O.decompress_rate(a2, 2), O.decompress(a))
    for sub in (False, True):
        got = O.add_rate(a2, b2, 2, sub=sub)
        ref = O.sub(a, b) if sub else O.add(a, b)
        assert np.array_equal(got.f, ref.f) and np.array_equal(got.s, ref.s)
        assert np.array_equal(got.phi, ref.phi) and np.array_equal(got.code, ref.code)
    # the 28-code order of the paper format is the rate-2 kept set
    assert [tuple(p) for p in O.kept_positions()] == kept_set(2)


def test_full_rate_codes_are_the_whole_truncated_dct():
    rng = np.random.default_rng(5)
    A = W.random_block_matrix(16, 24, seed=3)
    A[8:16, 0:8] = 2.5                     # a constant block
    A[0:8, 16:24] = rng.standard_normal((8, 8)) * 1e3
    c = O.compress_rate(A, 8)
    for b in range(c.nb):
        bi, bj = divmod(b, 3)
        st = O.block_stages(A[8 * bi:8 * bi + 8, 8 * bj:8 * bj + 8].copy())
        full = np.clip(np.trunc(st["dct"] * st["phi"]), -127, 127).astype(np.int8)
        assert np.array_equal(c.code[b], full.reshape(-1))
        assert c.phi[b] == st["phi"] and c.s[b] == st["s"] and c.f[b] == st["f"]


@pytest.mark.parametrize("kind", ["smooth", "noise", "wide"])
def test_codes_are_nested_across_rates(kind):
    A = W.random_block_matrix(32, 40, seed=9, kind=kind)
    B = W.random_block_matrix(32, 40, seed=10, kind=kind)
    full_a, full_b = O.compress_rate(A, 8), O.compress_rate(B, 8)
    sums = {s: O.add_rate(full_a, full_b, 8, sub=s) for s in (False, True)}
    for r in range(1, 8):
        idx = [i * 8 + j for i, j in kept_set(r)]
        a = O.compress_rate(A, r)
        assert np.array_equal(a.phi, full_a.phi) and np.array_equal(a.s, full_a.s)
        assert np.array_equal(a.code, full_a.code[:, idx])
        b = O.compress_rate(B, r)
        for s in (False, True):
            got = O.add_rate(a, b, r, sub=s)
            assert np.array_equal(got.code, sums[s].code[:, idx])
            assert np.array_equal(got.phi, sums[s].phi) and np.array_equal(got.f, sums[s].f)


def test_full_rate_round_trip_bound():
    """At r = 8 nothing is dropped and quantization is the only loss.  With X
    the block's DCT (from the pinned stage-by-stage oracle) and C its codes,
    the inverse DCT is orthonormal, so every delta is off by at most
    E = s ||X - C/phi||_2.  The inverse of the normalization carries
    e_0j = e_0,j-1 + err and e_ij = (e_i-1,j + e_i,j-1)/2 + err, so
    |e_ij| <= (i + j) E; and E < 8 s/phi since truncation leaves each
    coefficient within 1/phi."""
    A = np.concatenate([W.random_block_matrix(32, 32, seed=s, kind=k)
                        for s, k in ((1, "smooth"), (2, "noise"), (3, "smooth"))], axis=1)
    c = O.compress_rate(A, 8)
    Ah = O.decompress_rate(c, 8)
    nbc = A.shape[1] // 8
    ij = np.add.outer(np.arange(8), np.arange(8))
    used = 0.0
    for b in range(c.nb):
        bi, bj = divmod(b, nbc)
        blk = (slice(8 * bi, 8 * bi + 8), slice(8 * bj, 8 * bj + 8))
        st = O.block_stages(A[blk].copy())
        q = st["dct"] - c.code[b].reshape(8, 8).astype(float) / c.phi[b]
        assert np.all(np.abs(q) < 1.0 / c.phi[b])
        E = c.s[b] * np.linalg.norm(q)
        assert E < 8.0 * c.s[b] / c.phi[b]
        err = np.abs(Ah[blk] - A[blk])
        bound = ij * E * (1 + 1e-9) + 1e-13 * np.abs(A[blk]).max()
        assert np.all(err <= bound), (b, (err - bound).max())
        used = max(used, (err[ij > 0] / bound[ij > 0]).max())
    assert used > 0.3                        # the bound is not vacuous


def test_more_coefficients_lower_the_error_on_a_smooth_field():
    A, _ = W.plain_pair()
    errs = []
    for r in (1, 2, 4, 8):
        Ah = O.decompress_rate(O.compress_rate(A, r), r)
        errs.append(np.linalg.norm(Ah - A) / np.linalg.norm(A))
    assert errs[0] > errs[1] > errs[2] >= errs[3]
    assert errs[3] < 0.05



def test_rate_two_dots_and_products_are_the_paper_formats():
    """At r = 2 the rate-r dot, line x column and product equal the 28-code
    oracle's (pinned separately), within their own rounding."""
    A, Bm = W.plain_pair()
    a, b = O.compress_rate(A, 2), O.compress_rate(Bm, 2)
    v, av = O.dot_rate(a, b, 2)
    ref, aref = O.dot(O.compress(A), O.compress(Bm))
    assert abs(v - ref) <= 1e-14 * aref and abs(av - aref) <= 1e-14 * aref
    for i, j in ((17, 200), (0, 0), (255, 255)):
        v, av = O.dot_rowcol_rate(a, b, 2, i, j)
        ref, aref = O.dot_rowcol(O.compress(A), O.compress(Bm), i, j)
        assert abs(v - ref) <= 1e-14 * aref
    Bd = W.smoothed_normal(256, 40, seed=3)
    C, Cabs = O.matmul_rate(a, 2, Bd)
    assert np.all(np.abs(C - O.matmul(O.compress(A), Bd)) <= 1e-13 * Cabs)


def test_constant_blocks_make_the_dots_closed_form():
    """Blocks that are constant (K = 0: s = 0) decompress exactly at every
    rate, so <vec A_hat, vec B_hat> = 64 sum_b fa_b fb_b and line x column
    = sum over the k-blocks of 8 fa fb."""
    rng = np.random.default_rng(2)
    ca, cb = rng.standard_normal((4, 6)), rng.standard_normal((6, 3))
    A = np.kron(ca, np.ones((8, 8)))
    Bm = np.kron(cb, np.ones((8, 8)))
    A2 = np.kron(rng.standard_normal((4, 6)), np.ones((8, 8)))
    import math
    for r in (1, 3, 8):
        a, a2, b = O.compress_rate(A, r), O.compress_rate(A2, r), O.compress_rate(Bm, r)
        v, _ = O.dot_rate(a, a2, r)
        assert v == math.fsum(64.0 * x for x in (ca * A2[::8, ::8]).ravel())
        v, _ = O.dot_rowcol_rate(a, b, r, 9, 20)
        assert v == math.fsum(8.0 * ca[1, k] * cb[k, 2] for k in range(6))
        C, _ = O.matmul_rate(a, r, Bm)
        assert np.allclose(C, A @ Bm, rtol=1e-15, atol=0)


def test_worked_example_at_every_rate():
    """Sec. II, Example 5 prints all 64 re-scaled, truncated DCT values P' of
    the example block (the kept 28 and the one other nonzero entry, (4,4)
    1-indexed, that the 28-code format drops).  At rate r the stored codes
    must be those entries of P' in the rate's order; r = 4 keeps the (4,4)
    entry, and phi and f are the example's at every rate."""
    from conftest import load_golden

    g = load_golden("example_xy.txt")
    A = np.fromfunction(lambda i, j: (0.1 * i) * (0.1 * j), (8, 8))
    P1 = np.array([[int(x) for x in row] for row in g["P'"]])
    for r in range(1, 9):
        c = O.compress_rate(A, r)
        want = [P1[i, j] for i, j in kept_set(r)]
        assert list(c.code[0]) == want, r
        assert c.phi[0] == int(g["phi"][0][0]) and c.f[0] == float(g["f"][0][0])
    assert (3, 3) not in kept_set(3) and O.compress_rate(A, 4).code[0][kept_set(4).index((3, 3))] == 1
