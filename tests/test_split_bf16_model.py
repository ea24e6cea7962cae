"""Error model of the split-bf16 matrix product, emulated on the CPU, and the
discriminating power of the tolerances the GPU tests use.

The product splits A_hat and B into three bf16 slices each (X1 = RN_bf16(X),
X2 = RN_bf16(X - X1), X3 = RN_bf16(X - X1 - X2)) and sums the six slice
products of levels i + j <= 4 in fp32.  The emulation forms the same slices
and accumulates the same products in fp32 one term at a time, in the GEMM's
order of the inner dimension (the six slice products one after another).  It
checks that the full product meets both limits, and that a product missing
one level of slice products fails one of them:
  * the second-level pair A1 B2 + A2 B1 against SPLIT_BF16_LARGE_K_TOL at
    k = 1024 (random-signed terms of about 2^-9: errors around 3e-4);
  * the third-level triple A1 B3 + A2 B2 + A3 B1 against the worst-case bound
    split_bf16_tol(k) at k = 8 (at large k these terms, about 2^-18 each and
    random in sign, sit below the fp32 accumulation error, so only a small
    inner dimension can see them)."""
import numpy as np

import oracle as O
import workloads as W
from conftest import SPLIT_BF16_LARGE_K_TOL, split_bf16_tol

PAIRS = [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)]   # slice indexes, levels i + j + 2 = 2, 3, 3, 4, 4, 4


def bf16(x):
    """Round binary64 to bf16 (8 significant bits), to nearest, ties to even."""
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def slices(x):
    x1 = bf16(x)
    x2 = bf16(x - x1)
    return x1, x2, bf16(x - x1 - x2)


def split_product(A, Bm, levels):
    a, b = slices(A), slices(Bm)
    acc = np.zeros((A.shape[0], Bm.shape[1]), np.float32)
    for i, j in PAIRS:
        if i + j + 2 not in levels:
            continue
        for kk in range(A.shape[1]):
            # a bf16 x bf16 product is exact in fp32; the sum rounds
            acc = (acc + np.outer(a[i][:, kk], b[j][kk, :]).astype(np.float32)).astype(np.float32)
    return acc.astype(np.float64)


def componentwise(C, Ah, Bm):
    return float(np.max(np.abs(C - Ah @ Bm) / (np.abs(Ah) @ np.abs(Bm))))


def test_second_level_products_are_needed_at_large_k():
    k = 1024
    Ah = O.decompress(O.compress(W.bump_field(k, k)[:16]))
    Bm = W.smoothed_normal(k, k, seed=7)[:, :32]
    full = componentwise(split_product(Ah, Bm, (2, 3, 4)), Ah, Bm)
    no_second = componentwise(split_product(Ah, Bm, (2, 4)), Ah, Bm)
    assert full <= SPLIT_BF16_LARGE_K_TOL / 10
    assert no_second > 5 * SPLIT_BF16_LARGE_K_TOL


def test_third_level_products_are_needed_at_small_k():
    n, k, m = 64, 8, 64
    Ah = O.decompress(O.compress(W.random_block_matrix(n, k, seed=n + k)))
    Bm = W.smoothed_normal(k, m, seed=7)
    full = componentwise(split_product(Ah, Bm, (2, 3, 4)), Ah, Bm)
    no_third = componentwise(split_product(Ah, Bm, (2, 3)), Ah, Bm)
    assert full <= split_bf16_tol(k) / 2
    assert no_third > split_bf16_tol(k)
