"""Two fp32 decision rules of Algorithm 1, checked against the oracle at
every rate.

The rate-r addition uses the tiled 28-code kernel's rule (fp32 estimates of
beta_k, bound 1.25 2^-19 (...) + 2^-100); test_add_certification's numpy
emulation of that rule works on any number of codes per block and is reused
here on rate-r operands (test_rate_add_uses_the_tiled_rule).

The per-block addition kernel (used for unaligned code arrays) forms beta_1,
beta_2 exactly in binary64 as Algorithm 1 does, truncates them to fp32 and
decides each code from
    v = fl32(fma(b1f, c1, +-fl32(b2f c2))),
    E = 2^-21 fma(|b1f|, |c1|, fl32(|b2f| |c2|)) + 2^-22 |v| + 2^-100,
when [v - E, v + E] truncates to one code (or lies beyond +-127), and in
binary64 otherwise.  This test emulates that fp32 arithmetic in numpy (the
products of two fp32 numbers are exact in binary64; the fused multiply-add is
rounded once to binary64 and then to binary32) and checks every decided code
against the oracle's binary64 Algorithm 1 at every rate: pairs of compressed
fields, self-additions (v on integers), scaled partners and random slopes,
phi and codes over a wide exponent range."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from test_add_certification import kernel_codes

F32 = np.float32


def trunc32(x):
    """binary64 -> binary32 keeping the top 23 fraction bits (0 below the
    fp32 normal range)."""
    x = np.ascontiguousarray(x, np.float64)
    b = x.view(np.uint64) & np.uint64(0xFFFFFFFFE0000000)
    t = b.view(np.float64)
    return np.where(np.abs(t) < 2.0 ** -126, 0.0, t).astype(F32)


def fmaf(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def rate_codes(a, b, sub=False):
    """(codes, decided) of the fp32 path for out = a +- b."""
    ss = a.s + b.s
    pa, pb = a.phi.astype(np.int64), b.phi.astype(np.int64)
    ph = np.maximum(1, (pa * pb) // (pa + pb)).astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        b1 = (a.s / ss) / pa * ph
        b2 = (b.s / ss) / pb * ph
    e1 = (np.abs(b1).view(np.uint64) >> np.uint64(52)).astype(np.int64)
    e2 = (np.abs(b2).view(np.uint64) >> np.uint64(52)).astype(np.int64)
    fast = ((e1 < 1023 + 100) & (e2 < 1023 + 100))[:, None]
    b1f = trunc32(np.where(fast[:, 0], b1, 0.0))[:, None]
    b2f = trunc32(np.where(fast[:, 0], b2, 0.0))[:, None]
    x1, x2 = a.code.astype(F32), b.code.astype(F32)
    p2 = (b2f * x2).astype(F32)
    v = fmaf(b1f, x1, -p2 if sub else p2)
    inner = (np.abs(b2f) * np.abs(x2)).astype(F32)
    E = F32(2.0 ** -21) * fmaf(np.abs(b1f), np.abs(x1), inner)
    E = (E + F32(2.0 ** -22) * np.abs(v)).astype(F32) + F32(2.0 ** -100)
    lo, hi = (v - E).astype(F32), (v + E).astype(F32)
    code = np.where(lo >= 127, 127, np.where(hi <= -127, -127, np.trunc(lo)))
    decided = ((lo >= 127) | (hi <= -127) | (np.trunc(lo) == np.trunc(hi))) & fast
    zero_s = (ss == 0.0)[:, None]
    return np.where(zero_s, 0, code), decided | zero_s


def check(a, b, r, sub=False):
    ref = O.add_rate(a, b, r, sub=sub)
    code, decided = rate_codes(a, b, sub)
    bad = decided & (code != ref.code.astype(np.float64))
    assert not bad.any(), (np.argwhere(bad)[:5], code[bad][:5], ref.code[bad][:5])
    return 1.0 - decided.mean()


@pytest.mark.parametrize("r", [1, 2, 4, 8])
def test_rate_add_decisions_on_fields_and_self_additions(r):
    a = O.compress_rate(W.bump_field(256, 5, rows=128), r)
    b = O.compress_rate(W.bump_field(256, 6, rows=128), r)
    assert check(a, b, r) < 0.05 and check(a, b, r, sub=True) < 0.05
    s = a
    for _ in range(4):
        check(s, a, r)
        s = O.add_rate(s, a, r)
    for cst in (-0.97, -1.0, 3.5, 1e-300, 1e300):
        c = O.scale_rate(b, cst)
        check(a, c, r)
        check(a, c, r, sub=True)


def test_rate_add_decisions_on_random_slopes_phi_and_codes():
    rng = np.random.default_rng(77)
    n, r = 1 << 14, 8
    a, b = O.empty_rate(8, 8 * n, r), O.empty_rate(8, 8 * n, r)
    for m in (a, b):
        m.f[:] = rng.normal(size=n)
        m.s[:] = rng.choice([-1.0, 1.0], n) * np.exp(rng.uniform(-80, 80, n))
        m.phi[:] = rng.integers(1, 256, n)
        m.code[:] = rng.integers(-127, 128, (n, 64))
    b.s[: n // 8] = -a.s[: n // 8] * (1 + rng.uniform(-1e-12, 1e-12, n // 8))
    b.s[n // 8: n // 4] = a.s[n // 8: n // 4]
    b.s[n // 4: n // 4 + 64] = 0.0
    check(a, b, r)
    check(a, b, r, sub=True)


@pytest.mark.parametrize("r", [1, 2, 4, 8])
def test_rate_add_uses_the_tiled_rule(r):
    a = O.compress_rate(W.bump_field(256, 5, rows=128), r)
    b = O.compress_rate(W.bump_field(256, 6, rows=128), r)
    pairs = [(a, b), (a, a), (O.add_rate(a, a, r), a)] + [(a, O.scale_rate(b, c)) for c in (-0.97, -1.0, 1e-300, 1e300)]
    worst = 0.0
    for n_pair, (x, y) in enumerate(pairs):
        for sub in (False, True):
            ref = O.add_rate(x, y, r, sub=sub)
            for p1 in (-1.0, 0.0, 1.0):
                for p2 in (-1.0, 0.0, 1.0):
                    code, decided = kernel_codes(x, y, p1, p2, sub)
                    bad = decided & (code != ref.code.astype(np.float64))
                    assert not bad.any(), (np.argwhere(bad)[:5], code[bad][:5], ref.code[bad][:5])
                    if n_pair < 3:   # beyond: partners scaled out of the fp32 beta range go to binary64
                        worst = max(worst, 1.0 - decided.mean())
    assert worst < 0.5
