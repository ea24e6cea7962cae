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
// <= sum |D'| < K + 1 (every |cos_kx| <= 1).  The kernel uses
//     E_ij = 24u aa_ij (K + 1) + 2^-100.
#pragma once

#include "block_codec.cuh"
#include "exact_div.cuh"
#include "gmap.cuh"

namespace blaz {

// x * 0.5 rounded to nearest even, on the bit pattern (no FP64 instruction):
// an exponent decrement for normal results; for the smallest normals and the
// subnormals the significand is halved with round-half-even; Inf and NaN
// are returned as they are (NaN blocks take the exact path anyway).
__device__ __forceinline__ double dhalf(double x)
{
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e > 1 && e < 0x7FF) return __longlong_as_double(b - (1ll << 52));
    if (e == 0x7FF) return x;
    const unsigned long long sign = (unsigned long long)b & 0x8000000000000000ull;
    unsigned long long m = (unsigned long long)b & 0x000FFFFFFFFFFFFFull;
    if (e == 1) m |= 1ull << 52;
    unsigned long long q = m >> 1;
    if ((m & 1ull) && (q & 1ull)) q += 1ull;
    return __longlong_as_double((long long)(sign | q));
}

// trunc toward zero saturated to [-127, 127], NaN -> 0 (quantize), on the bits.
__device__ __forceinline__ int8_t quantize_bits(double v)
{
    const long long b = __double_as_longlong(v);
    const bool neg = b < 0;
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0x7FF) return (b & 0x000FFFFFFFFFFFFFll) ? 0 : (neg ? -127 : 127);
    if (e < 1023) return 0;
    if (e >= 1023 + 7) return neg ? -127 : 127;
    const unsigned long long m = ((unsigned long long)b & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    int mag = (int)(m >> (52 - (e - 1023)));
    mag = mag > 127 ? 127 : mag;
    return (int8_t)(neg ? -mag : mag);
}

// Exact float -> double on the bits (normal floats and zero).
__device__ __forceinline__ double f2d_bits(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xFF;
    if (e == 0) return 0.0;
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e - 127 + 1023) << 52) |
                                 ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
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
// non-increasing in m.  The comparison and truncation act on the bits.
__device__ __forceinline__ int phi_of(double m)
{
    const double q = ddiv(127.0, m);
    const long long b = __double_as_longlong(q);
    const int e = (int)((b >> 52) & 0x7FF);
    if (b < 0) return 1;                 // negative (not reached: m >= 0)
    if (e >= 1023 + 8) return 255;       // q >= 256, Inf, NaN
    if (e < 1023) return 1;              // q < 1
    const unsigned long long mm = ((unsigned long long)b & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    const int p = (int)(mm >> (52 - (e - 1023)));
    return p >= 255 ? 255 : p;
}

// Non-negative doubles compare as their bit patterns.
__device__ __forceinline__ double dmax_nonneg(double a, double b)
{
    return __double_as_longlong(a) >= __double_as_longlong(b) ? a : b;
}

// 1 when x != 0 (NaN included), 0 for +-0, on the integer pipe: the OR of
// the magnitude bits goes through inline PTX so that the compiler cannot
// fold the test back into a binary64 comparison.
__device__ __forceinline__ int nonzero_bits(double x)
{
    unsigned m;
    asm("or.b32 %0, %1, %2;" : "=r"(m) : "r"((unsigned)__double2hiint(x) << 1), "r"((unsigned)__double2loint(x)));
    return m != 0u;
}

// s = RN(S/K) for the nonzero count 1 <= K <= 64 (exact_div.cuh).
__device__ __forceinline__ double div_by_count(double S, int K) { return div_small_int(S, K); }

constexpr uint32_t kPendingAll = 0x80000000u;  // phi not certified / non-finite: whole block exact

// Compress one block held in d (overwritten).  Returns 0 when every decision
// is certified (s, phi and the codes set); kPendingAll when the block must go
// through compress_block; otherwise a mask of the codes (bit t = code t) left
// undecided, with s, phi and the other codes set.  s_out is always exact.
__device__ __forceinline__ uint32_t compress_block_fast(double (&d)[64], double &s_out, uint8_t &phi_out,
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
    // Eqs. eqslope, eqslope2 (K counted on the bit patterns: x != 0; S as the
    // pairwise tree).
    int K = 0;
#pragma unroll
    for (int p = 0; p < 64; ++p) K += nonzero_bits(d[p]);
    const double S = tree_sum_abs(d);
    if (K == 0) {
        s_out = 0.0;
        phi_out = 255;
#pragma unroll
        for (int t = 0; t < kKeep; ++t) code[t] = 0;
        return 0u;
    }
    const double s = div_by_count(S, K);
    const double r = ddiv(1.0, s);
    s_out = s;
    // Inf / NaN / overflow (S >= 0, r >= 0): exact path
    if (((__double_as_longlong(S) >> 52) & 0x7FF) >= 0x7FE || ((__double_as_longlong(r) >> 52) & 0x7FF) >= 0x7FE)
        return kPendingAll;

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
    // E_ij / aa_ij, one factor for the block.
    const float base = 24.0f * 0x1p-24f * (float)(K + 1);
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
    // phi = trunc(RN(127/m)) in [1, 255] is decided in fp32 from bounds
    // m_lo <= m <= m_hi: the quotients 127/m_hi, 127/m_lo (correctly rounded,
    // widened by 2^-20) bound the real 127/m, whose binary64 rounding moves
    // it by 2^-53 relative, so equal clamped truncations at both ends fix
    // phi.  When the other coefficients are certainly below |X00|, m = |X00|
    // exactly and an undecided phi takes the exact division.
    const double ax00 = fabs(X00);
    const float a00 = trunc_f32(ax00);                  // a00 <= |X00| < a00 (1 + 2^-23)
    const bool m_exact = __double_as_longlong(f2d_bits(mhi * (1.0f + 0x1p-20f))) < __double_as_longlong(ax00);
    const float m_lo = m_exact ? a00 : fmaxf(a00, mlo * (1.0f - 0x1p-20f));
    const float m_hi = m_exact ? a00 * (1.0f + 0x1p-22f) : fmaxf(a00 * (1.0f + 0x1p-22f), mhi * (1.0f + 0x1p-20f));
    const float q_lo = __fdiv_rn(127.0f, m_hi) * (1.0f - 0x1p-20f);
    const float q_hi = __fdiv_rn(127.0f, m_lo) * (1.0f + 0x1p-20f);
    const int p_lo = q_lo >= 255.0f ? 255 : (q_lo < 1.0f ? 1 : (int)q_lo);
    const int p_hi = q_hi >= 255.0f ? 255 : (q_hi < 1.0f ? 1 : (int)q_hi);
    int phi = p_lo;
    if (p_lo != p_hi) {
        if (!m_exact) return kPendingAll;
        phi = phi_of(ax00);
    }
    phi_out = (uint8_t)phi;
    const float phif = (float)phi;
    code[0] = quantize_bits(dmul(X00, i64_to_double(phi)));
    uint32_t pending = 0u;
#pragma unroll
    for (int t = 1; t < kKeep; ++t) {
        const float aa = (float)aa_tab(kept_row(t), kept_col(t));
        const float v = Dk[t] * phif;
        const float Ev = (base * aa * phif) * (1.0f + 0x1p-20f) + 0x1p-22f * (fabsf(v) + 1.0f) + 0x1p-16f;
        const float lo = v - Ev, hi = v + Ev;
        int c = 0;
        if (lo >= 127.0f) c = 127;
        else if (hi <= -127.0f) c = -127;
        else {
            const int tl = (int)truncf(lo), th = (int)truncf(hi);
            if (tl != th || tl >= 127 || tl <= -127) pending |= 1u << t;
            else c = tl;
        }
        code[t] = (int8_t)c;
    }
    return pending;
}

// ---------------------------------------------------------------------------
// Two-phase form of the certified compressor, for the two-kernel path, where
// the exact DC chain runs only for the blocks that need it.
//
// The DC code is X00 phi truncated, X00 = RN(aa00 * U00) with U00 the
// binary64 sums of D' in the specified order.  For a sign-coherent block (all
// nonzero D of one sign) sum D' = +-K exactly, so X00 phi sits on an integer
// whenever 8 | K phi and only the exact binary64 value decides it: such
// blocks get the exact chain.  For the others the DC is one more fp32
// coefficient under the bound below, and an undecided DC code goes to the
// fix-up like any other code.
//
// Rows in fp32 from D and r directly: with e the exponent of s, D 2^-e and
// r 2^e are exact (power-of-two scaling) and of order 1; both are truncated
// to fp32 (relative error < 2u each, u = 2^-24) and multiplied in fp32 (u):
// |D'_f - D'| <= 5u |D'| + 2^-126 against D' = RN64(D r), so the first term
// of the bound in the header becomes 5u and E_ij = 28u aa_ij (K + 1) + 2^-100
// covers the total of 25u + O(u^2).

// binary64 -> binary32 of x 2^-e by truncating the significand (x 2^-e < 2^127);
// values below 2^-126 (after scaling) and subnormal x become 0.
__device__ __forceinline__ float trunc_f32_scaled(double x, int e)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int ex = (int)((hi >> 20) & 0x7FF);
    const int ef = ex - 1023 - e + 127;
    if (ex == 0 || ef <= 0) return 0.0f;
    const unsigned mant = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
    return __uint_as_float((hi & 0x80000000u) | ((unsigned)ef << 23) | mant);
}

// What the first phase leaves for the second.
struct FastCtx {
    uint32_t state;     // 0: decide in cf_finish; kPendingAll: whole block exact; 1: done (K == 0)
    bool coherent;      // sign-coherent: the exact X00 comes from the dense DC pass
    float base;         // E_ij / aa_ij
    float mlo, mhi;     // bounds on max |X| over the 63 coefficients other than the DC
    float Dk[kKeep];    // fp32 kept coefficients (Dk[0]: the DC estimate)
};

// Phase 1: normalization, slope (both exact), fp32 DCT of all 64
// coefficients.  d holds D afterwards (the dense DC pass reads it).
__device__ __forceinline__ void cf_prepare(double (&d)[64], double &s_out, double &r_out, FastCtx &c)
{
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
    int K = 0;
    unsigned pos = 0u, neg = 0u;  // any nonzero D of each sign
#pragma unroll
    for (int p = 0; p < 64; ++p) {
        const int nz = nonzero_bits(d[p]);
        K += nz;
        const unsigned sg = (unsigned)__double2hiint(d[p]) >> 31;
        pos |= (unsigned)nz & (sg ^ 1u);
        neg |= (unsigned)nz & sg;
    }
    c.coherent = false;
    r_out = 0.0;
    if (K == 0) {
        s_out = 0.0;
        c.state = 1u;
        return;
    }
    const double S = tree_sum_abs(d);
    const double s = div_by_count(S, K);
    const double r = ddiv(1.0, s);
    s_out = s;
    r_out = r;
    const int es_field = (int)((__double_as_longlong(s) >> 52) & 0x7FF);
    // Inf / NaN / overflow, or a subnormal s: exact path
    if (((__double_as_longlong(S) >> 52) & 0x7FF) >= 0x7FE || ((__double_as_longlong(r) >> 52) & 0x7FF) >= 0x7FE ||
        es_field == 0) {
        c.state = kPendingAll;
        return;
    }
    c.state = 0u;
    c.coherent = (pos ^ neg) != 0u;
    const int e = es_field - 1023;
    const float rr = trunc_f32_scaled(r, -e);
    float T[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        float rf[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) rf[v] = trunc_f32_scaled(d[u * 8 + v], e) * rr;
        float t0 = rf[0];
#pragma unroll
        for (int v = 1; v < 8; ++v) t0 += rf[v];
        T[u][0] = t0;
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            float acc = rf[0] * cos_f(j, 0);
#pragma unroll
            for (int v = 1; v < 8; ++v) acc = fmaf(rf[v], cos_f(j, v), acc);
            T[u][j] = acc;
        }
    }
    c.base = 28.0f * 0x1p-24f * (float)(K + 1);
    float mlo = 0.0f, mhi = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float acc = cos_f(i, 0) * T[0][j];
#pragma unroll
            for (int u = 1; u < 8; ++u) acc = fmaf(cos_f(i, u), T[u][j], acc);
            const float aa = (float)aa_tab(i, j);
            const float Df = aa * acc;
            if (!(i == 0 && j == 0)) {
                const float E = c.base * aa + 1e-30f;
                const float a = fabsf(Df);
                mhi = fmaxf(mhi, a + E);
                mlo = fmaxf(mlo, a - E);
            }
            const int t = kept_index(i, j);
            if (t >= 0) c.Dk[t] = Df;
        }
    }
    c.mlo = mlo;
    c.mhi = mhi;
}

// The exact DC coefficient X00 = RN(aa00 U00) from D and r (the dense pass).
__device__ __forceinline__ double cf_exact_dc(const double *D, double r)
{
    double U00 = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        double t0 = dmul(D[u * 8], r);
#pragma unroll
        for (int v = 1; v < 8; ++v) t0 = dadd(t0, dmul(D[u * 8 + v], r));
        U00 = (u == 0) ? t0 : dadd(U00, t0);
    }
    return dmul(BLAZ_A00, U00);
}

// Phase 2: phi and the codes, with the exact X00 of a coherent block.
// Returns 0, kPendingAll or the mask of undecided codes (as
// compress_block_fast).
__device__ __forceinline__ uint32_t cf_finish(const FastCtx &c, double X00, uint8_t &phi_out, int8_t (&code)[kKeep])
{
    if (c.state == 1u) {
        phi_out = 255;
#pragma unroll
        for (int t = 0; t < kKeep; ++t) code[t] = 0;
        return 0u;
    }
    if (c.state == kPendingAll) return kPendingAll;
    // bounds on m = max(|X00|, the others), as in compress_block_fast; for a
    // non-coherent block |X00| is itself known to within E00
    const float aa00 = (float)BLAZ_A00;
    const float E00 = c.base * aa00 + 1e-30f;
    bool m_exact = false;
    double ax00 = 0.0;
    float dc_lo, dc_hi;
    if (c.coherent) {
        ax00 = fabs(X00);
        const float a00 = trunc_f32(ax00);
        m_exact = __double_as_longlong(f2d_bits(c.mhi * (1.0f + 0x1p-20f))) < __double_as_longlong(ax00);
        dc_lo = a00;
        dc_hi = a00 * (1.0f + 0x1p-22f);
    } else {
        const float a = fabsf(c.Dk[0]);
        dc_lo = fmaxf(0.0f, (a - E00) * (1.0f - 0x1p-20f));
        dc_hi = (a + E00) * (1.0f + 0x1p-20f);
    }
    const float m_lo = m_exact ? dc_lo : fmaxf(dc_lo, c.mlo * (1.0f - 0x1p-20f));
    const float m_hi = m_exact ? dc_hi : fmaxf(dc_hi, c.mhi * (1.0f + 0x1p-20f));
    const float q_lo = __fdiv_rn(127.0f, m_hi) * (1.0f - 0x1p-20f);
    const float q_hi = __fdiv_rn(127.0f, m_lo) * (1.0f + 0x1p-20f);
    const int p_lo = q_lo >= 255.0f ? 255 : (q_lo < 1.0f ? 1 : (int)q_lo);
    const int p_hi = q_hi >= 255.0f ? 255 : (q_hi < 1.0f ? 1 : (int)q_hi);
    int phi = p_lo;
    if (p_lo != p_hi) {
        if (!m_exact) return kPendingAll;
        phi = phi_of(ax00);
    }
    phi_out = (uint8_t)phi;
    const float phif = (float)phi;
    uint32_t pending = 0u;
#pragma unroll
    for (int t = 0; t < kKeep; ++t) {
        if (t == 0 && c.coherent) {
            code[0] = quantize_bits(dmul(X00, i64_to_double(phi)));
            continue;
        }
        const float aa = (float)aa_tab(kept_row(t), kept_col(t));
        const float v = c.Dk[t] * phif;
        const float Ev = (c.base * aa * phif) * (1.0f + 0x1p-20f) + 0x1p-22f * (fabsf(v) + 1.0f) + 0x1p-16f;
        const float lo = v - Ev, hi = v + Ev;
        int cc = 0;
        if (lo >= 127.0f) cc = 127;
        else if (hi <= -127.0f) cc = -127;
        else {
            const int tl = (int)truncf(lo), th = (int)truncf(hi);
            if (tl != th || tl >= 127 || tl <= -127) pending |= 1u << t;
            else cc = tl;
        }
        code[t] = (int8_t)cc;
    }
    return pending;
}

// cos and alpha_i alpha_j as tables for run-time indices (the exact fix-up).
__constant__ double c_cos[64] = {
#define BLAZ_ROW(k) cos_tab(k, 0), cos_tab(k, 1), cos_tab(k, 2), cos_tab(k, 3), cos_tab(k, 4), cos_tab(k, 5), cos_tab(k, 6), cos_tab(k, 7)
    BLAZ_ROW(0), BLAZ_ROW(1), BLAZ_ROW(2), BLAZ_ROW(3), BLAZ_ROW(4), BLAZ_ROW(5), BLAZ_ROW(6), BLAZ_ROW(7)
#undef BLAZ_ROW
};

// Code t of a block from the exact D' (binary64 order of the specification):
// T[u] = sum_v D'[u][v] cos[j][v], U = sum_u cos[i][u] T[u], X = aa_ij U,
// code = quantize(X * phi).
__device__ __forceinline__ int8_t exact_code(const double (&dp)[64], int t, int phi)
{
    const int i = kept_row(t), j = kept_col(t);
    double U = 0.0;
    for (int u = 0; u < 8; ++u) {
        double T = (j == 0) ? dp[u * 8] : dmul(dp[u * 8], c_cos[j * 8]);
#pragma unroll
        for (int v = 1; v < 8; ++v) T = dadd(T, (j == 0) ? dp[u * 8 + v] : dmul(dp[u * 8 + v], c_cos[j * 8 + v]));
        const double term = (i == 0) ? T : dmul(c_cos[i * 8 + u], T);
        U = (u == 0) ? term : dadd(U, term);
    }
    const double aa = (i == 0 && j == 0) ? BLAZ_A00 : (i == 0 || j == 0) ? BLAZ_A0K : BLAZ_AKK;
    return quantize_bits(dmul(dmul(aa, U), i64_to_double(phi)));
}

// D' = D * (1/s) of a block in d (input block on entry), as compress_block
// forms it; s is the block's exact stored slope (> 0).
__device__ __forceinline__ void exact_dprime(double (&d)[64], double s)
{
#pragma unroll
    for (int i = 7; i >= 0; --i) {
#pragma unroll
        for (int j = 7; j >= 0; --j) {
            if (i == 0 && j == 0) d[0] = 0.0;
            else if (i == 0) d[j] = dsub(d[j], d[j - 1]);
            else if (j == 0) d[i * 8] = dsub(d[i * 8], d[(i - 1) * 8]);
            else d[i * 8 + j] = dhalf(dadd(dsub(d[i * 8 + j], d[(i - 1) * 8 + j]), dsub(d[i * 8 + j], d[i * 8 + j - 1])));
        }
    }
    const double r = ddiv(1.0, s);
#pragma unroll
    for (int p = 0; p < 64; ++p) d[p] = dmul(d[p], r);
}

}  // namespace blaz
