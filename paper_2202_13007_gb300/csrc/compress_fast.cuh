// compress_fast.cuh -- the compressor of Sec. II of "Compressed Matrix
// Computations" (arXiv 2202.13007) with most of the DCT moved off the FP64
// pipe, while every stored bit stays identical to the binary64 operation
// order of include/blaz.h (the order compress_block in block_codec.cuh
// evaluates).
//
// The stored values are f, s, phi and 28 truncated codes.  f and s need the
// exact normalized block, so the normalization, slope and reciprocal run in
// binary64 as specified.  The DCT matters only through the truncations that
// make phi and the codes, so it is evaluated in fp32 with a proven error
// bound, and a decision is taken only when the whole interval allowed by the
// bound truncates to one value.  The DC coefficient is different: for
// sign-coherent blocks its real value sits exactly on an integer code
// (K/8 * phi), so its binary64 value -- 0.125 times the row-major sums of
// D' in the specified order -- is always computed exactly.  A block where
// some decision is not certified is left to the exact path.
//
// Error bound (u = 2^-24).  With D'_f the truncation of the exact binary64
// D' (relative error < 2u), c_f = RN32(cos) (error <= u|c|), fp32 FMA chains
// of 8 terms (error <= gamma_8 of the sum of |terms|) in both passes and
// aa_f = RN32(alpha_i alpha_j), the fp32 coefficient D_f satisfies
//     |D_f - X| <= (2u + u + 8u + u + 8u + 2u + O(u^2)) aa_ij S2_ij + 2^-100
// against the binary64 coefficient X of the specification, whose own error
// (17 roundings of 2^-53) is far below u; S2_ij = sum_uv |c_iu c_jv D'_uv|
// <= sum |D'| < K + 1.  The kernel uses E_ij = 32u aa_ij (K+1) + 2^-100.
#pragma once

#include "block_codec.cuh"

namespace blaz {

// x * 0.5 rounded to nearest: an exponent decrement for normal numbers with a
// biased exponent >= 2 (exact), and zero kept as is; the binary64 multiply
// for everything else (subnormals, the smallest normals, Inf, NaN).
__device__ __forceinline__ double dhalf(double x)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int e = (hi >> 20) & 0x7FF;
    if (e > 1 && e < 0x7FF) return __hiloint2double(hi - (1 << 20), lo);
    if (((hi & 0x7FFFFFFF) | lo) == 0) return x;
    return dmul(x, 0.5);
}

// binary64 -> binary32 by truncating the significand: relative error < 2^-23
// for |x| >= 2^-126; smaller values become 0.  Requires finite |x| < 2^127.
__device__ __forceinline__ float trunc_f32(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7FF) - 1023 + 127;
    if (e <= 0) return 0.0f;
    const unsigned mant = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
    return __uint_as_float((hi & 0x80000000u) | ((unsigned)e << 23) | mant);
}

__host__ __device__ constexpr float cos_f(int k, int x) { return (float)cos_tab(k, x); }

// phi of Eq. eqphi from m: trunc(RN(127/m)) clamped to [1, 255]; monotone
// non-increasing in m.
__device__ __forceinline__ int phi_of(double m)
{
    const double q = ddiv(127.0, m);
    if (!(q < 255.0)) return 255;
    const int p = __double2int_rz(q);
    return p < 1 ? 1 : p;
}

// Compress one block held in d (overwritten).  Returns true with s, phi and
// the codes set when every decision is certified; false when the block must
// go through compress_block.  s_out is the exact s in both cases.
__device__ __forceinline__ bool compress_block_fast(double (&d)[64], double &s_out, uint8_t &phi_out,
                                                    int8_t (&code)[kKeep])
{
    // Eq. eqnorm, exactly as compress_block (x * 0.5 by dhalf, bit-identical).
#pragma unroll
    for (int i = 7; i >= 0; --i) {
#pragma unroll
        for (int j = 7; j >= 0; --j) {
            if (i == 0 && j == 0) {
                d[0] = 0.0;
            } else if (i == 0) {
                d[j] = dsub(d[j], d[j - 1]);
            } else if (j == 0) {
                d[i * 8] = dsub(d[i * 8], d[(i - 1) * 8]);
            } else {
                const double a = dsub(d[i * 8 + j], d[(i - 1) * 8 + j]);
                const double b = dsub(d[i * 8 + j], d[i * 8 + j - 1]);
                d[i * 8 + j] = dhalf(dadd(a, b));
            }
        }
    }
    // Eqs. eqslope, eqslope2 (K counted on the bit patterns: x != 0).
    int K = 0;
    double S = 0.0;
#pragma unroll
    for (int p = 0; p < 64; ++p) {
        K += (__double_as_longlong(d[p]) << 1) != 0;
        S = dadd(S, fabs(d[p]));
    }
    if (K == 0) {
        s_out = 0.0;
        phi_out = 255;
#pragma unroll
        for (int t = 0; t < kKeep; ++t) code[t] = 0;
        return true;
    }
    const double s = ddiv(S, (double)K);
    const double r = ddiv(1.0, s);
    s_out = s;
    if (!(S <= 1.7e308) || !(r <= 1.7e308)) return false;  // Inf / NaN / overflow: exact path

    // Rows of D' (exact binary64), the exact inner sums of column 0 (the DC
    // chain, cos(0) = 1) and fp32 inner sums T[u][j] for j >= 1.
    float T[8][8];
    double U00 = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        double row[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) row[v] = dmul(d[u * 8 + v], r);
        double t0 = row[0];
#pragma unroll
        for (int v = 1; v < 8; ++v) t0 = dadd(t0, row[v]);
        U00 = (u == 0) ? t0 : dadd(U00, t0);
        float rf[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) rf[v] = trunc_f32(row[v]);
        T[u][0] = trunc_f32(t0);
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            float acc = rf[0] * cos_f(j, 0);
#pragma unroll
            for (int v = 1; v < 8; ++v) acc = fmaf(rf[v], cos_f(j, v), acc);
            T[u][j] = acc;
        }
    }
    const double X00 = dmul(BLAZ_A00, U00);

    // Outer sums in fp32; bounds on max |X| over the other 63 coefficients.
    const float base = 32.0f * 0x1p-24f * (float)(K + 1);
    float Dk[kKeep];
    float mlo = 0.0f, mhi = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i == 0 && j == 0) continue;
            float acc = cos_f(i, 0) * T[0][j];
#pragma unroll
            for (int u = 1; u < 8; ++u) acc = fmaf(cos_f(i, u), T[u][j], acc);
            const float aa = (float)aa_tab(i, j);
            const float Df = aa * acc;
            const float E = base * aa + 1e-30f;
            const float a = fabsf(Df);
            mhi = fmaxf(mhi, a + E);
            mlo = fmaxf(mlo, a - E);
            const int t = kept_index(i, j);
            if (t >= 0) Dk[t] = Df;
        }
    }
    // Eq. eqphi.  m = max(|X00|, max over the others), certified when phi is
    // the same at both ends of the interval of possible m.
    const double ax00 = fabs(X00);
    const double mhi_d = (double)mhi * (1.0 + 0x1p-20);
    const double mlo_d = (double)mlo * (1.0 - 0x1p-20);
    int phi;
    if (mhi_d < ax00) {
        phi = phi_of(ax00);  // the DC coefficient is the maximum: m is exact
    } else {
        const int p_lo_m = phi_of(fmax(ax00, mlo_d));
        const int p_hi_m = phi_of(fmax(ax00, mhi_d));
        if (p_lo_m != p_hi_m) return false;
        phi = p_hi_m;
    }
    phi_out = (uint8_t)phi;
    const float phif = (float)phi;
    code[0] = quantize(dmul(X00, (double)phi));
#pragma unroll
    for (int t = 1; t < kKeep; ++t) {
        const float aa = (float)aa_tab(kept_row(t), kept_col(t));
        const float v = Dk[t] * phif;
        const float Ev = (base * aa * phif) * (1.0f + 0x1p-20f) + 0x1p-22f * (fabsf(v) + 1.0f) + 0x1p-16f;
        const float lo = v - Ev, hi = v + Ev;
        int c;
        if (lo >= 127.0f) c = 127;
        else if (hi <= -127.0f) c = -127;
        else {
            const int tl = (int)truncf(lo), th = (int)truncf(hi);
            if (tl != th || tl >= 127 || tl <= -127) return false;
            c = tl;
        }
        code[t] = (int8_t)c;
    }
    return true;
}

}  // namespace blaz
