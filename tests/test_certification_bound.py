"""The certified compressor decides phi and the codes from fp32 estimates of
the DCT coefficients and an error bound E_ij; a decision is only as sound as
the bound.  This test evaluates the fp32 estimates exactly as the fast
kernel forms them (numpy emulation: truncations to fp32, RN32 products,
fused multiply-adds as one rounding of the exact product plus the addend,
the same summation order) and checks |D_f - X| <= E_ij against the binary64
coefficients X of the oracle, on random blocks and on blocks built to make
the fp32 error large (long same-sign sums, wide dynamic range, few nonzeros).

Three forms of the estimate are checked:
  * rows from the exact D' = RN64(D r), truncated to fp32, E = 24u aa (K+1);
  * rows from D 2^-e truncated to fp32 times the row scale
    rr = RN32(1 / trunc32(s 2^-e)) (e the exponent of s; within 3u of
    2^e RN64(1/s)), multiplied in fp32, E = 28u aa (K+1);
  * the uniform-block form: D 2^-e rounded to nearest in fp32 (the kernel
    converts the integer N of D = N 2^k to fp32 and scales it by a power of
    two, which is exact), times the same rr, E = 28u aa (K+1);
with u = 2^-24 and an absolute 2^-100.  The first form runs 8-term fp32
chains in both passes; the other two, as the certified kernels, sums and
differences of mirrored entries (the DCT basis is even or odd under
x -> 7 - x) feeding 4-term chains."""
import numpy as np
import pytest

import oracle as O

F32 = np.float32
U = 2.0 ** -24


def trunc32(x):
    """binary64 -> binary32 truncating the significand (values below 2^-126 -> 0)."""
    x = np.float64(x)
    if x == 0.0 or abs(x) < 2.0 ** -126:
        return F32(0.0)
    b = np.array([x]).view(np.uint64)[0]
    b &= np.uint64(0xFFFFFFFFE0000000)          # keep 23 fraction bits
    return F32(np.array([b], dtype=np.uint64).view(np.float64)[0])


def fma32(a, b, c):
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def estimates(d, r, s, K, scaled):
    cos, aa = O.dct_tables()
    cf = cos.astype(F32)
    rows = np.zeros((8, 8), F32)
    if scaled:
        e = int(np.frexp(s)[1]) - 1               # s = m 2^e, 1 <= m < 2
        rr = F32(1.0) / trunc32(np.ldexp(s, -e))    # RN32 of the reciprocal of an fp32
        for u in range(8):
            for v in range(8):
                x = F32(np.ldexp(d[u, v], -e)) if scaled == "uniform" else trunc32(np.ldexp(d[u, v], -e))
                rows[u, v] = F32(np.float64(x) * np.float64(rr))
    else:
        for u in range(8):
            for v in range(8):
                rows[u, v] = trunc32(np.float64(d[u, v]) * np.float64(r))
    T = np.zeros((8, 8), F32)
    D = np.zeros((8, 8), np.float64)
    if not scaled:
        # 8-term chains in both passes (the one-kernel form)
        for u in range(8):
            t0 = rows[u, 0]
            for v in range(1, 8):
                t0 = F32(t0 + rows[u, v])
            T[u, 0] = t0
            for j in range(1, 8):
                acc = F32(rows[u, 0] * cf[j, 0])
                for v in range(1, 8):
                    acc = fma32(rows[u, v], cf[j, v], acc)
                T[u, j] = acc
        for j in range(8):
            for i in range(8):
                acc = F32(cf[i, 0] * T[0, j])
                for u in range(1, 8):
                    acc = fma32(cf[i, u], T[u, j], acc)
                D[i, j] = F32(F32(aa[i, j]) * acc)
        return D, aa
    # the certified passes: sums and differences of mirrored entries (cos_jx
    # is even or odd in x -> 7 - x with j) feeding 4-term chains
    for u in range(8):
        sv = [F32(rows[u, v] + rows[u, 7 - v]) for v in range(4)]
        dv = [F32(rows[u, v] - rows[u, 7 - v]) for v in range(4)]
        t0 = sv[0]
        for v in range(1, 4):
            t0 = F32(t0 + sv[v])
        T[u, 0] = t0
        for j in range(1, 8):
            x = dv if j % 2 else sv
            acc = F32(x[0] * cf[j, 0])
            for v in range(1, 4):
                acc = fma32(x[v], cf[j, v], acc)
            T[u, j] = acc
    for j in range(8):
        S = [F32(T[u, j] + T[7 - u, j]) for u in range(4)]
        Dd = [F32(T[u, j] - T[7 - u, j]) for u in range(4)]
        for i in range(8):
            x = Dd if i % 2 else S
            acc = F32(cf[i, 0] * x[0])
            for u in range(1, 4):
                acc = fma32(cf[i, u], x[u], acc)
            D[i, j] = F32(F32(aa[i, j]) * acc)
    return D, aa


def adversarial_blocks(rng):
    yield np.add.outer(np.arange(8.0), np.arange(8.0))                          # all D equal: long same-sign sums
    yield np.add.outer(np.arange(8.0) ** 2, np.arange(8.0) * 3)                 # growing same-sign D
    b = np.zeros((8, 8)); b[7, 7] = 1.0; yield b                                # one nonzero pattern
    yield np.cumsum(np.cumsum(rng.uniform(0, 1, (8, 8)), 0), 1)                 # sign-coherent, smooth
    yield rng.standard_normal((8, 8)) * 10.0 ** rng.integers(-8, 8, (8, 8))     # wide dynamic range
    yield np.add.outer(np.arange(8.0), np.arange(8.0)) * 1e-300                 # tiny scale
    yield np.add.outer(np.arange(8.0), np.arange(8.0)) * 1e300                  # huge scale
    for k in range(1, 8):
        yield np.fromfunction(lambda i, j: np.cos(np.pi * (2 * j + 1) * k / 16) * np.cos(np.pi * (2 * i + 1) * k / 16),
                              (8, 8)).cumsum(0).cumsum(1)                       # energy in one coefficient


@pytest.mark.parametrize("scaled", [False, True, "uniform"])
def test_fp32_estimates_are_within_the_certification_bound(scaled):
    rng = np.random.default_rng(2026)
    blocks = list(adversarial_blocks(rng))
    blocks += [rng.standard_normal((8, 8)) for _ in range(60)]
    blocks += [np.cumsum(np.cumsum(rng.standard_normal((8, 8)), 0), 1) for _ in range(60)]
    factor = 28.0 if scaled else 24.0
    checked = 0
    for M in blocks:
        st = O.block_stages(M)
        K = st["K"]
        s = st["s"]
        if K == 0 or not np.isfinite(s) or s == 0.0 or s < 2.0 ** -1022:
            continue
        r = 1.0 / s
        if not np.isfinite(r):
            continue
        D, aa = estimates(st["delta"], r, s, K, scaled)
        X = st["dct"]
        E = factor * U * aa * (K + 1) + 2.0 ** -100
        assert np.all(np.abs(D - X) <= E), (np.max(np.abs(D - X) / E), M)
        checked += 1
    assert checked >= 120
