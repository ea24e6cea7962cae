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
// Rows in fp32 from D and s directly: with e the exponent of s, D 2^-e is
// exact (power-of-two scaling) and of order 1 and is truncated to fp32
// (relative error < 2u, u = 2^-24); the row scale rr = RN32(1 /
// trunc32(s 2^-e)) is within 3u of 2^e RN64(1/s) (a truncation below 2u, one
// correctly rounded fp32 reciprocal, the binary64 rounding far below); one
// fp32 product (u): |D'_f - D'| <= 6u |D'| + 2^-126 against D' = RN64(D r)
// with r = RN64(1/s), so the first term of the bound in the header becomes 6u
// and E_ij = 28u aa_ij (K + 1) + 2^-100 covers the total of 26u + O(u^2).
// The exact r is formed only for the blocks whose exact DC chain needs it
// (sign-coherent blocks, by the block's lane after its DCT), off every
// block's path to the DCT.  Both passes of this form add and subtract mirrored entries first
// (cos_kx is even or odd under x -> 7 - x, exactly in the table) and run
// 4-term chains: one rounding of |a| + |b| and gamma_4 of the chain stay
// within the 8u per pass that the bound allows for 8-term chains.

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

// Eq. eqnorm in place with binary64 operations, from the last element
// backwards (M(i-1,j) and M(i,j-1) are still inputs when D(i,j) is formed);
// the interior halving x * 0.5 is dhalf (bit-identical, integer pipe).
__device__ __forceinline__ void normalize_block(double (&d)[64])
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
}

// Uniform blocks.  When the 64 entries of a block share one sign and one
// exponent field e (54 <= e <= 2045), each is m 2^(e-1075) with an integer
// significand m in [2^52, 2^53), and every operation of Eq. eqnorm is exact:
// M_ij - M_i-1,j = (m - m') 2^(e-1075) with |m - m'| < 2^52, the sum of two
// such differences stays below 2^53 units, and the halving of a normal
// number is exact.  So D_ij = N_ij 2^(e-1076) with the integer
//     N_ij = 2 m_ij - m_i-1,j - m_i,j-1  (interior),  2 (m_ij - m_prev) (row 0, column 0),
// |N| < 2^53, which the integer pipe forms without any rounding.  If
// moreover sum |N| < 2^53, every partial sum of the pairwise |D| tree is a
// multiple of 2^(e-1076) below 2^53 of them, so each of its binary64
// additions is exact and S = (sum |N|) 2^(e-1076) whatever the order.
// e >= 54 keeps every D and S a normal number or an exact multiple of the
// smallest subnormal; e <= 2045 keeps them finite.
__device__ __forceinline__ bool block_is_uniform(const double (&d)[64])
{
    const unsigned h0 = (unsigned)__double2hiint(d[0]);
    const unsigned e = (h0 >> 20) & 0x7FFu;
    // the OR of hi(M) ^ hi(M00) over the block (one three-input logic
    // operation per entry) is below 2^20 iff all share sign and exponent
    unsigned diff = 0u;
#pragma unroll
    for (int p = 1; p < 64; ++p) diff |= (unsigned)__double2hiint(d[p]) ^ h0;
    return diff < (1u << 20) && e >= 54u && e <= 2045u;
}

// a 2^(e-1076) with the given sign bit, for 0 < a < 2^53 and 54 <= e <= 2045
// (exact; a normal number); +0 for a == 0.
__device__ __forceinline__ double scaled_int_to_double(unsigned long long a, unsigned long long sign, int e)
{
    const int lz = __clzll((long long)a);  // >= 11
    // leading one shifted to bit 52 carries into the exponent field: e + 9 - lz + 1
    const unsigned long long bits = (sign << 63) | (((unsigned long long)(e + 9 - lz) << 52) + (a << ((lz - 11) & 63)));
    return a ? __longlong_as_double((long long)bits) : 0.0;
}

// The integer form of Eq. eqnorm for a uniform block: d holds the input on
// entry and the integers N (as bit patterns) on exit.  The significands are
// magnitudes, so for a block of negative entries D = -N 2^(e-1076); a zero
// D is +0, as the binary64 difference of equal values is (uniform_d gives
// the binary64 D, bit-identical to normalize_block).  Returns sum |N|
// (exact), and K, pos, neg as the caller's count loop would.
__device__ __forceinline__ unsigned long long normalize_uniform(double (&d)[64], int e, unsigned bneg, int &K,
                                                                unsigned &pos, unsigned &neg)
{
    auto sig = [&](int p) -> long long {
        return (long long)(((unsigned long long)__double_as_longlong(d[p]) & 0x000FFFFFFFFFFFFFull) |
                           0x0010000000000000ull);
    };
    // sum N telescopes to the boundary: row 0 and column 0 give
    // 2 (m_07 - m_00) + 2 (m_70 - m_00); the interior's column differences
    // give sum_j>0 (m_7j - m_0j) and its row differences sum_i>0 (m_i7 - m_i0)
    long long tot = 2 * ((sig(7) - sig(0)) + (sig(56) - sig(0)));
#pragma unroll
    for (int q = 1; q < 8; ++q) tot += (sig(56 + q) - sig(q)) + (sig(q * 8 + 7) - sig(q * 8));
#pragma unroll
    for (int i = 7; i >= 0; --i) {
#pragma unroll
        for (int j = 7; j >= 0; --j) {
            long long N;
            if (i == 0 && j == 0) N = 0;
            else if (i == 0) N = 2 * (sig(j) - sig(j - 1));
            else if (j == 0) N = 2 * (sig(i * 8) - sig((i - 1) * 8));
            else N = 2 * sig(i * 8 + j) - sig((i - 1) * 8 + j) - sig(i * 8 + j - 1);
            d[i * 8 + j] = __longlong_as_double(N);  // the integer, until converted below
        }
    }
    // sum |N| = 2 sum_{N>0} N - sum N; all nonzero N have one sign iff
    // |sum N| = sum |N|
    long long psum = 0;
    K = 0;
#pragma unroll
    for (int p = 0; p < 64; ++p) {
        const long long N = __double_as_longlong(d[p]);
        psum += N > 0 ? N : 0ll;
        K += (int)(N != 0ll);
    }
    const unsigned long long sum = (unsigned long long)(2 * psum - tot);
    const bool coherent = (unsigned long long)(tot < 0 ? -tot : tot) == sum;
    // as the caller's flags would be: D has the sign of N, flipped for a negative block
    const unsigned tneg = (unsigned)((unsigned long long)tot >> 63) ^ bneg;
    pos = K && (!coherent || !tneg) ? 1u : 0u;
    neg = K && (!coherent || tneg) ? 1u : 0u;
    return sum;
}

// D = N 2^(e-1076) with the block's sign (bneg) as binary64 (exact).
__device__ __forceinline__ double uniform_d(long long N, int e, unsigned bneg)
{
    const unsigned long long a = N < 0 ? (unsigned long long)(-N) : (unsigned long long)N;
    return scaled_int_to_double(a, (unsigned long long)(((unsigned)((unsigned long long)N >> 63)) ^ bneg), e);
}

// Phase 1, after the normalization (K nonzero entries, pos / neg: any
// nonzero D of each sign; S = sum |D| when K > 0): slope, the fp32 row scale
// and the fp32 DCT of all 64 coefficients.  kInt: d holds the integers N of a
// uniform block with exponent field eb (D = +-N 2^(eb-1076)); otherwise d
// holds D.  d is left as it is.
template <bool kInt>
__device__ __forceinline__ void cf_slope_and_dct(const double (&d)[64], int eb, unsigned bneg, int K, unsigned pos,
                                                 unsigned neg, double S, double &s_out, FastCtx &c)
{
    c.coherent = false;
    if (K == 0) {
        s_out = 0.0;
        c.state = 1u;
        return;
    }
    const double s = div_by_count(S, K);
    s_out = s;
    const int es_field = (int)((__double_as_longlong(s) >> 52) & 0x7FF);
    // Inf / NaN / overflow, or a subnormal s: exact path (a normal s has a
    // finite normal 1/s)
    if (((__double_as_longlong(S) >> 52) & 0x7FF) >= 0x7FE || es_field == 0) {
        c.state = kPendingAll;
        return;
    }
    c.state = 0u;
    c.coherent = (pos ^ neg) != 0u;
    const int e = es_field - 1023;
    const float rr = __frcp_rn(trunc_f32_scaled(s, e));  // 2^e / s within 3u
    // Both passes run two independent chains per instruction on the paired
    // fp32 pipe of sm_103a (__fmul2_rn, __fadd2_rn, __ffma2_rn round each
    // lane as the scalar operation does, so every coefficient is the same
    // chain of 8 fp32 operations as before): rows u, u + 1 in the first pass,
    // coefficients (i, j), (i + 1, j) in the second.
    // The rows D 2^-e (1/s) 2^e in fp32.  From D: both factors truncated to
    // fp32 (2u each) and one fp32 product (u).  From N (kInt): RN32(N) (u)
    // times rr 2^(eb-1076-e), a power-of-two scaling of the truncated rr
    // (exact: the exponent stays within about 60 of zero) and by the block's
    // sign, one product (u).  Both stay within the 5u relative error of the
    // bound in the header.
    const float rr_int = kInt ? __int_as_float((int)(bneg << 31) | ((127 + eb - 1076 - e) << 23)) * rr : 0.0f;
    float2 T[4][8];  // T[u / 2][j] = (T_u,j, T_u+1,j)
#pragma unroll
    for (int up = 0; up < 4; ++up) {
        const float2 rr2 = kInt ? make_float2(rr_int, rr_int) : make_float2(rr, rr);
        float2 rf[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const double x0 = d[2 * up * 8 + v], x1 = d[(2 * up + 1) * 8 + v];
            const float2 in = kInt ? make_float2(__ll2float_rn(__double_as_longlong(x0)),
                                                 __ll2float_rn(__double_as_longlong(x1)))
                                   : make_float2(trunc_f32_scaled(x0, e), trunc_f32_scaled(x1, e));
            rf[v] = __fmul2_rn(in, rr2);
        }
        // cos_jx is even in x -> 7 - x for even j and odd for odd j, exactly
        // (the table is built so), so each row's sums and differences of
        // mirrored entries feed 4-term chains (error below 5u of the sum of
        // |terms|, against gamma_8 for the 8-term chains the bound allows)
        float2 sv[4], dv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            sv[v] = __fadd2_rn(rf[v], rf[7 - v]);
            dv[v] = __ffma2_rn(rf[7 - v], make_float2(-1.0f, -1.0f), rf[v]);  // rf_v - rf_7-v, one rounding
        }
        float2 t0 = sv[0];
#pragma unroll
        for (int v = 1; v < 4; ++v) t0 = __fadd2_rn(t0, sv[v]);
        T[up][0] = t0;
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            const float2 *x = (j & 1) ? dv : sv;
            float2 acc = __fmul2_rn(x[0], make_float2(cos_f(j, 0), cos_f(j, 0)));
#pragma unroll
            for (int v = 1; v < 4; ++v) acc = __ffma2_rn(x[v], make_float2(cos_f(j, v), cos_f(j, v)), acc);
            T[up][j] = acc;
        }
    }
    c.base = 28.0f * 0x1p-24f * (float)(K + 1);
    float max0k = 0.0f, maxkk = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float Dij[8];
        // the same symmetry over u: (T_u + T_7-u, T_u - T_7-u) in one paired
        // operation, the sum for the even output row i0 and the difference
        // for the odd one i1 of each pair
        float2 SD[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float Tu = (u & 1) ? T[u / 2][j].y : T[u / 2][j].x;
            const float Tm = ((7 - u) & 1) ? T[(7 - u) / 2][j].y : T[(7 - u) / 2][j].x;
            SD[u] = __ffma2_rn(make_float2(Tm, Tm), make_float2(1.0f, -1.0f), make_float2(Tu, Tu));
        }
#pragma unroll
        for (int ip = 0; ip < 4; ++ip) {
            const int i0 = 2 * ip, i1 = 2 * ip + 1;
            float2 acc = __fmul2_rn(make_float2(cos_f(i0, 0), cos_f(i1, 0)), SD[0]);
#pragma unroll
            for (int u = 1; u < 4; ++u) acc = __ffma2_rn(make_float2(cos_f(i0, u), cos_f(i1, u)), SD[u], acc);
            const float2 D2 = __fmul2_rn(make_float2((float)aa_tab(i0, j), (float)aa_tab(i1, j)), acc);
            Dij[i0] = D2.x;
            Dij[i1] = D2.y;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float Df = Dij[i];
            // the largest |D_f| per alpha_i alpha_j class (E_ij depends on the
            // class only; fp32 addition is monotone, so adding E to the
            // class maximum gives the maximum of |D_f| + E and of |D_f| - E)
            if (i == 0 && j == 0) {
            } else if (i == 0 || j == 0) {
                max0k = fmaxf(max0k, fabsf(Df));
            } else {
                maxkk = fmaxf(maxkk, fabsf(Df));
            }
            const int t = kept_index(i, j);
            if (t >= 0) c.Dk[t] = Df;
        }
    }
    const float E0k = c.base * (float)BLAZ_A0K + 1e-30f, Ekk = c.base * (float)BLAZ_AKK + 1e-30f;
    c.mhi = fmaxf(max0k + E0k, maxkk + Ekk);
    c.mlo = fmaxf(fmaxf(max0k - E0k, maxkk - Ekk), 0.0f);
}

// Phase 1 on the binary64 pipe: Eq. eqnorm, the nonzero count and the
// pairwise |D| tree as specified, then cf_slope_and_dct.  stash(d, meta) is
// called between the two for a block whose nonzero D all have one sign (the
// dense DC pass will need D: the caller keeps a copy, or in the uniform pass
// only the block's index), so that d can die row by row in the DCT.
template <typename Stash>
__device__ __forceinline__ void cf_prepare(double (&d)[64], double &s_out, FastCtx &c, Stash stash)
{
    normalize_block(d);
    int K = 0;
    unsigned pos = 0u, neg = 0u;
#pragma unroll
    for (int p = 0; p < 64; ++p) {
        const int nz = nonzero_bits(d[p]);
        K += nz;
        const unsigned sg = (unsigned)__double2hiint(d[p]) >> 31;
        pos |= (unsigned)nz & (sg ^ 1u);
        neg |= (unsigned)nz & sg;
    }
    if (K && (pos ^ neg)) stash(d, 0u);
    cf_slope_and_dct<false>(d, 0, 0u, K, pos, neg, K ? tree_sum_abs(d) : 0.0, s_out, c);
}

// Phase 1 for a uniform block on the integer pipe (same bits as
// cf_prepare).  d holds the integers N on success (meta: the exponent field
// and the block's sign for uniform_d).  Returns false, with d no longer the
// input, when the block is not uniform or its |N| sum could round: such
// blocks take cf_prepare.  stash as in cf_prepare (d then holds N).
template <typename Stash>
__device__ __forceinline__ bool cf_prepare_uniform(double (&d)[64], double &s_out, FastCtx &c, Stash stash)
{
    if (!block_is_uniform(d)) return false;
    const unsigned hi0 = (unsigned)__double2hiint(d[0]);
    const int e = (int)((hi0 >> 20) & 0x7FFu);
    const unsigned bneg = hi0 >> 31;
    int K;
    unsigned pos, neg;
    const unsigned long long sum = normalize_uniform(d, e, bneg, K, pos, neg);
    if (sum >= (1ull << 53)) return false;
    if (K && (pos ^ neg)) stash(d, (unsigned)e | (bneg << 16));
    cf_slope_and_dct<true>(d, e, bneg, K, pos, neg, scaled_int_to_double(sum, 0ull, e), s_out, c);
    return true;
}

// The exact DC coefficient X00 = RN(aa00 U00) from D and r.
__device__ __forceinline__ double cf_exact_dc(const double *D, double r)
{
    double U00 = 0.0;
    // rows not unrolled: D is in shared memory, and a short loop keeps this
    // rarely run code small in the instruction cache
#pragma unroll 1
    for (int u = 0; u < 8; ++u) {
        double t0 = dmul(D[u * 8], r);
#pragma unroll
        for (int v = 1; v < 8; ++v) t0 = dadd(t0, dmul(D[u * 8 + v], r));
        U00 = (u == 0) ? t0 : dadd(U00, t0);
    }
    return dmul(BLAZ_A00, U00);
}

// The same X00 by a team of 8 lanes, lane u holding row u of D (drow(v) =
// D_uv) and r = RN(1/s): the row chains t_u = sum_v RN(D_uv r) (v
// ascending) are independent, and lane 0 of the team adds them in the
// specified order (u ascending) from the team's shuffles, so the chain is
// ~16 binary64 operations deep instead of ~130.  Same bits as cf_exact_dc.
// Returns X00 in lane 0 of the team.
template <typename Row>
__device__ __forceinline__ double cf_exact_dc_rows(Row drow, double r, unsigned tmask, int tbase)
{
    double t = dmul(drow(0), r);
#pragma unroll
    for (int v = 1; v < 8; ++v) t = dadd(t, dmul(drow(v), r));
    double U00 = __shfl_sync(tmask, t, tbase);
#pragma unroll
    for (int uu = 1; uu < 8; ++uu) U00 = dadd(U00, __shfl_sync(tmask, t, tbase + uu));
    return dmul(BLAZ_A00, U00);
}

// X00 by a team from D in shared memory (the binary64 pass).
__device__ __forceinline__ double cf_exact_dc_team(const double *D, double r, int u, unsigned tmask, int tbase)
{
    return cf_exact_dc_rows([&](int v) { return D[u * 8 + v]; }, r, tmask, tbase);
}

// X00 by a team for a uniform block from its integers N in shared memory
// (meta as cf_prepare_uniform sets it).
__device__ __forceinline__ double cf_exact_dc_team_n(const double *N, double r, unsigned meta, int u, unsigned tmask,
                                                     int tbase)
{
    const int e = (int)(meta & 0xFFFFu);
    const unsigned bneg = meta >> 16;
    return cf_exact_dc_rows([&](int v) { return uniform_d(__double_as_longlong(N[u * 8 + v]), e, bneg); }, r, tmask,
                            tbase);
}

// X00 by a team for a uniform block b (meta as cf_prepare_uniform sets it)
// from the input itself: lane u reloads rows u and u - 1 of the block
// (clamped to the rows x cols matrix as load_block_clamped is) and forms row
// u of the integers N as normalize_uniform does, then the exact D =
// uniform_d(N).  The block's own lane has just loaded these rows (an L1 or
// L2 hit), and the CTA keeps no copy of the block.
__device__ __forceinline__ double cf_exact_dc_team_uniform(const double *__restrict__ A, int64_t lda, int64_t rows,
                                                           int64_t cols, int64_t nbc, int64_t b, double r,
                                                           unsigned meta, int u, unsigned tmask, int tbase)
{
    const int64_t bi = b / nbc, bj = b - (b / nbc) * nbc;
    const int64_t row = bi * 8 + u < rows ? bi * 8 + u : rows - 1;
    const int64_t rowp = bi * 8 + u - 1 < rows ? bi * 8 + u - 1 : rows - 1;  // read for u > 0 only
    auto sig = [](double x) -> long long {
        return (long long)(((unsigned long long)__double_as_longlong(x) & 0x000FFFFFFFFFFFFFull) |
                           0x0010000000000000ull);
    };
    long long cur[8], prev[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const int64_t c = bj * 8 + v < cols ? bj * 8 + v : cols - 1;
        cur[v] = sig(__ldg(A + row * lda + c));
        prev[v] = u > 0 ? sig(__ldg(A + rowp * lda + c)) : 0ll;
    }
    const int e = (int)(meta & 0xFFFFu);
    const unsigned bneg = meta >> 16;
    return cf_exact_dc_rows(
        [&](int v) {
            long long N;
            if (u == 0) N = v == 0 ? 0ll : 2 * (cur[v] - cur[v - 1]);
            else if (v == 0) N = 2 * (cur[0] - prev[0]);
            else N = 2 * cur[v] - prev[v] - cur[v - 1];
            return uniform_d(N, e, bneg);
        },
        r, tmask, tbase);
}

// Phase 2: phi and the codes, with the exact X00 of a coherent block.
// Returns 0, kPendingAll or the mask of undecided codes (as
// compress_block_fast).
__device__ __forceinline__ uint32_t cf_finish(const FastCtx &c, double X00, uint8_t &phi_out, uint32_t (&cw)[7])
{
    if (c.state == 1u) {
        phi_out = 255;
#pragma unroll
        for (int q = 0; q < 7; ++q) cw[q] = 0u;
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
    // Each code from the interval v -+ Ev, v = D_f phi, with
    // Ev = E_ij phi (1 + 2^-20) + 2^-22 (|v| + 1) + 2^-16 (the last two
    // terms cover the fp32 roundings of v and of the interval ends); two
    // codes per paired fp32 instruction, one constant per alpha class.
    auto cls = [&](int t) {
        const float aa = (float)aa_tab(kept_row(t), kept_col(t));
        return (c.base * aa * phif) * (1.0f + 0x1p-20f) + (0x1p-22f + 0x1p-16f);
    };
    const float C00 = cls(0), C0k = cls(1), Ckk = cls(9);
    auto cst = [&](int t) {
        const int i = kept_row(t), j = kept_col(t);
        return (i == 0 && j == 0) ? C00 : (i == 0 || j == 0) ? C0k : Ckk;
    };
    // A code is decided when the saturating int8 truncations of both ends
    // agree and are not -128 (below quantize's -127): the same decisions as
    // the truncations of both ends saturated to +-127 agreeing, except that
    // an interval reaching below -128 goes to the fix-up.  Four codes per
    // word, compared at once (undecided_bytes); bit t of the returned mask:
    // code t.
    const float2 phi2 = make_float2(phif, phif), k22 = make_float2(0x1p-22f, 0x1p-22f),
                 neg1 = make_float2(-1.0f, -1.0f);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        uint32_t l8[4], h8[4];
#pragma unroll
        for (int k = 0; k < 4; k += 2) {
            const int t0 = 4 * q + k, t1 = t0 + 1;
            const float2 v = __fmul2_rn(make_float2(c.Dk[t0], c.Dk[t1]), phi2);
            const float2 Ev = __ffma2_rn(make_float2(fabsf(v.x), fabsf(v.y)), k22, make_float2(cst(t0), cst(t1)));
            const float2 lo = __ffma2_rn(Ev, neg1, v), hi = __fadd2_rn(v, Ev);
            l8[k] = cvt_s8_rz(lo.x);
            l8[k + 1] = cvt_s8_rz(lo.y);
            h8[k] = cvt_s8_rz(hi.x);
            h8[k + 1] = cvt_s8_rz(hi.y);
        }
        const uint32_t lw = __byte_perm(__byte_perm(l8[0], l8[1], 0x0040), __byte_perm(l8[2], l8[3], 0x0040), 0x5410);
        const uint32_t hw = __byte_perm(__byte_perm(h8[0], h8[1], 0x0040), __byte_perm(h8[2], h8[3], 0x0040), 0x5410);
        cw[q] = lw;
        // bits 7, 15, 23, 31 of the byte mask to bits 28..31, then to 4q..4q+3
        pending |= ((undecided_bytes(lw, hw) * 0x00204081u) >> 28) << (4 * q);
    }
    if (c.coherent) {  // the DC of a sign-coherent block from its exact X00
        cw[0] = (cw[0] & 0xFFFFFF00u) | (uint32_t)(uint8_t)quantize_bits(dmul(X00, i64_to_double(phi)));
        pending &= ~1u;
    }
    return pending;
}

// cos and alpha_i alpha_j as tables for run-time indices (the exact fix-up).
__constant__ double c_cos[64] = {
#define BLAZ_ROW(k) cos_tab(k, 0), cos_tab(k, 1), cos_tab(k, 2), cos_tab(k, 3), cos_tab(k, 4), cos_tab(k, 5), cos_tab(k, 6), cos_tab(k, 7)
    BLAZ_ROW(0), BLAZ_ROW(1), BLAZ_ROW(2), BLAZ_ROW(3), BLAZ_ROW(4), BLAZ_ROW(5), BLAZ_ROW(6), BLAZ_ROW(7)
#undef BLAZ_ROW
};

}  // namespace blaz
