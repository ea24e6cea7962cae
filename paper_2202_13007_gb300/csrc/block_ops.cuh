// block_ops.cuh -- per-block device code of the operations on compressed
// blocks, shared by the standalone kernels and the persistent batch kernel:
// addition / subtraction (Algorithm 1, Eq. eq55 of "Compressed Matrix
// Computations", arXiv 2202.13007) and multiplication by a constant
// (Algorithm 2).  Bit-exact binary64 (explicit round-to-nearest intrinsics).
#pragma once

#include "blaz_internal.cuh"
#include "exact_div.cuh"

namespace blaz {

// Block b of out = a +- b.  Every input of the block is read before anything
// is written, so out may alias a or b.
template <bool kSub>
__device__ __forceinline__ void add_block(int64_t b, const double *f1, const double *s1, const uint8_t *p1,
                                          const int8_t *c1, const double *f2, const double *s2, const uint8_t *p2,
                                          const int8_t *c2, double *f, double *s, uint8_t *p, int8_t *c)
{
    const double fa = f1[b], fb = f2[b], sa = s1[b], sb = s2[b];
    const int pa = p1[b], pb = p2[b];
    uint32_t wa[7], wb[7];
    const uint32_t *ca = reinterpret_cast<const uint32_t *>(c1 + b * kKeep);
    const uint32_t *cb = reinterpret_cast<const uint32_t *>(c2 + b * kKeep);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        wa[q] = ca[q];
        wb[q] = cb[q];
    }
    const double fs = kSub ? dsub(fa, fb) : dadd(fa, fb);
    const double ss = dadd(sa, sb);
    int ph = (pa * pb) / (pa + pb);
    ph = ph < 1 ? 1 : ph;
    uint32_t wo[7];
    if (ss == 0.0) {
#pragma unroll
        for (int q = 0; q < 7; ++q) wo[q] = 0u;
    } else {
        const double a1 = ddiv(sa, ss);
        const double a2 = ddiv(sb, ss);
        // beta_k = (alpha_k / phi_k) phi: division by the integer phi_k without
        // a division sequence, integers converted on the integer pipe
        const double phd = i64_to_double(ph);
        const double b1 = dmul(div_small_int(a1, pa), phd);
        const double b2 = dmul(div_small_int(a2, pb), phd);
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            uint32_t v = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double x1 = (double)(int8_t)(uint8_t)(wa[q] >> (8 * k));
                const double x2 = (double)(int8_t)(uint8_t)(wb[q] >> (8 * k));
                const double y = kSub ? dsub(dmul(b1, x1), dmul(b2, x2)) : dadd(dmul(b1, x1), dmul(b2, x2));
                v |= (uint32_t)(uint8_t)quantize(y) << (8 * k);
            }
            wo[q] = v;
        }
    }
    f[b] = fs;
    s[b] = ss;
    p[b] = (uint8_t)ph;
    uint32_t *co = reinterpret_cast<uint32_t *>(c + b * kKeep);
#pragma unroll
    for (int q = 0; q < 7; ++q) co[q] = wo[q];
}

// Block b of out = cst * a (Algorithm 2); phi and codes copied when out != a.
__device__ __forceinline__ void scale_block(int64_t b, const double *f1, const double *s1, const uint8_t *p1,
                                            const int8_t *c1, double cst, double *f, double *s, uint8_t *p,
                                            int8_t *c, bool copy)
{
    f[b] = dmul(f1[b], cst);
    s[b] = dmul(s1[b], cst);
    if (copy) {
        p[b] = p1[b];
        const uint32_t *src = reinterpret_cast<const uint32_t *>(c1 + b * kKeep);
        uint32_t *dst = reinterpret_cast<uint32_t *>(c + b * kKeep);
#pragma unroll
        for (int q = 0; q < 7; ++q) dst[q] = src[q];
    }
}

// Block b of out = a +- b with the 28 code decisions taken in fp32 where a
// proven bound certifies them; bit-identical to add_block.
//   Spec:  y = RN64(RN64(b1 c1) +- RN64(b2 c2)),  code = trunc(y) saturated.
//   fp32:  v = fl(fl(b1f c1) +- b2f c2) (one product rounded, one fma), with
//          b1f, b2f the truncations of b1, b2 (relative error < 2^-23).
//   |v - y| <= (2u + 2u + u + 2^-29)(|b1 c1| + |b2 c2|) < 6u (|b1f c1| + |b2f c2|)
//   with u = 2^-24; a code is decided in fp32 when [v - E, v + E] truncates
//   to one value, otherwise it is evaluated exactly as in add_block.
__device__ __forceinline__ float small_int_to_float(int c) { return __int_as_float(0x4B400000 + c) - 12582912.0f; }

__device__ __forceinline__ float trunc_to_f32(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7FF) - 1023 + 127;
    if (e <= 0) return 0.0f;
    if (e >= 255) return __uint_as_float((hi & 0x80000000u) | 0x7F800000u);  // Inf (not used when finite)
    const unsigned mant = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
    return __uint_as_float((hi & 0x80000000u) | ((unsigned)e << 23) | mant);
}

template <bool kSub>
__device__ __forceinline__ void add_block_fast(int64_t b, const double *f1, const double *s1, const uint8_t *p1,
                                               const int8_t *c1, const double *f2, const double *s2,
                                               const uint8_t *p2, const int8_t *c2, double *f, double *s,
                                               uint8_t *p, int8_t *c)
{
    const double fa = f1[b], fb = f2[b], sa = s1[b], sb = s2[b];
    const int pa = p1[b], pb = p2[b];
    uint32_t wa[7], wb[7];
    const uint32_t *ca = reinterpret_cast<const uint32_t *>(c1 + b * kKeep);
    const uint32_t *cb = reinterpret_cast<const uint32_t *>(c2 + b * kKeep);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        wa[q] = ca[q];
        wb[q] = cb[q];
    }
    const double fs = kSub ? dsub(fa, fb) : dadd(fa, fb);
    const double ss = dadd(sa, sb);
    int ph = (pa * pb) / (pa + pb);
    ph = ph < 1 ? 1 : ph;
    uint32_t wo[7];
    if (ss == 0.0) {
#pragma unroll
        for (int q = 0; q < 7; ++q) wo[q] = 0u;
    } else {
        const double a1 = ddiv(sa, ss);
        const double a2 = ddiv(sb, ss);
        // beta_k = (alpha_k / phi_k) phi: division by the integer phi_k without
        // a division sequence, integers converted on the integer pipe
        const double phd = i64_to_double(ph);
        const double b1 = dmul(div_small_int(a1, pa), phd);
        const double b2 = dmul(div_small_int(a2, pb), phd);
        const unsigned e1 = ((unsigned)__double2hiint(b1) >> 20) & 0x7FF, e2 = ((unsigned)__double2hiint(b2) >> 20) & 0x7FF;
        // fp32 path for finite |b| < 2^100 (no Inf / NaN / overflow in fp32)
        const bool fast = e1 < 1023 + 100 && e2 < 1023 + 100;
        const float b1f = trunc_to_f32(b1), b2f = trunc_to_f32(b2);
        const float ab1 = fabsf(b1f), ab2 = fabsf(b2f);
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            uint32_t v32 = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i1 = (int)(int8_t)(uint8_t)(wa[q] >> (8 * k));
                const int i2 = (int)(int8_t)(uint8_t)(wb[q] >> (8 * k));
                const float x1 = small_int_to_float(i1), x2 = small_int_to_float(i2);
                int code = 0;
                bool done = false;
                if (fast) {
                    const float v = fmaf(b1f, x1, kSub ? -(b2f * x2) : b2f * x2);
                    const float E = 0x1p-21f * fmaf(ab1, fabsf(x1), ab2 * fabsf(x2)) + 0x1p-22f * fabsf(v) + 0x1p-100f;
                    const float lo = v - E, hi = v + E;
                    if (lo >= 127.0f) { code = 127; done = true; }
                    else if (hi <= -127.0f) { code = -127; done = true; }
                    else {
                        const int tl = (int)truncf(lo), th = (int)truncf(hi);
                        if (tl == th) { code = tl; done = true; }
                    }
                }
                if (!done) {
                    const double x1d = (double)i1, x2d = (double)i2;
                    const double y = kSub ? dsub(dmul(b1, x1d), dmul(b2, x2d)) : dadd(dmul(b1, x1d), dmul(b2, x2d));
                    code = quantize(y);
                }
                v32 |= (uint32_t)(uint8_t)(int8_t)code << (8 * k);
            }
            wo[q] = v32;
        }
    }
    f[b] = fs;
    s[b] = ss;
    p[b] = (uint8_t)ph;
    uint32_t *co = reinterpret_cast<uint32_t *>(c + b * kKeep);
#pragma unroll
    for (int q = 0; q < 7; ++q) co[q] = wo[q];
}

// fp32 estimate of beta_k = RN(RN(RN(s_k / s) / phi_k) * phi) (Algorithm 1)
// for the tiled addition (k_blockops.cu) and the rate-r addition (k_rate.cu);
// rho = phi / phi_k, evaluated in fp32.
//   s_k and s are truncated to fp32 after scaling both by 2^-e(s) (exponent
//   arithmetic on the integer pipe, exact): relative error < 2^-23 each;
//   __fdividef: < 2^-22; rho: < 2^-22; the product: < 2^-24.  So
//   |beta - beta_k| < (2^-21 + 2^-22 + 2^-24)(1 + 2^-20) |beta_k| < 2^-20 |beta_k|
//   (the three binary64 roundings of beta_k are below 2^-51 relative).
// s_k == 0 gives beta = 0 exactly (beta_k is a signed zero).  Returns false
// when s_k or s is subnormal, Inf or NaN, or when |s_k / s| leaves
// [2^-100, 2^101): the caller then evaluates beta_k in binary64.
__device__ __forceinline__ bool beta_f32(double sk, double ss, float rho, float &beta)
{
    const unsigned hk = (unsigned)__double2hiint(sk), lk = (unsigned)__double2loint(sk);
    const unsigned hs = (unsigned)__double2hiint(ss), ls = (unsigned)__double2loint(ss);
    if (((hk & 0x7FFFFFFFu) | lk) == 0u) {
        beta = 0.0f;
        return true;
    }
    const int ek = (int)((hk >> 20) & 0x7FF), es = (int)((hs >> 20) & 0x7FF);
    const int d = ek - es;
    if (ek == 0 || ek == 0x7FF || es == 0 || es == 0x7FF || d < -100 || d > 100) return false;
    const float xk = __uint_as_float((hk & 0x80000000u) | ((unsigned)(d + 127) << 23) |
                                     (__funnelshift_l(lk, hk, 3) & 0x7FFFFFu));
    const float xs = __uint_as_float((hs & 0x80000000u) | (127u << 23) | (__funnelshift_l(ls, hs, 3) & 0x7FFFFFu));
    beta = __fmul_rn(__fdividef(xk, xs), rho);
    return true;
}

}  // namespace blaz
