// k_dot.cu -- dot products on compressed matrices ("Dot product", Sec. III of
// "Compressed Matrix Computations", arXiv 2202.13007):
//   * the flattened product <vec A_hat, vec B_hat> of two same-shape matrices;
//   * Algorithm 3 (Eqs. eqbbb0, eqbbb): line i of A_hat times column j of B_hat.
// Reductions follow a fixed tree, so results are bitwise reproducible run to
// run.
//
// The flattened product never decompresses.  Decompression is linear in the
// codes: a block is A_hat = f 1 + t G c with t = s/phi and G the fixed 64 x 28
// map from codes to the block (inverse DCT of the kept coefficients followed
// by the inverse of Eq. eqnorm).  Hence, per block,
//     <A_hat, B_hat> = 64 fa fb + fa tb w.cb + fb ta w.ca + ta tb ca^T H cb,
// with w = G^T 1 and H = G^T G.  H and w are split into five fixed-point
// slices of 11 bits (integer digits times powers of two); with integer codes
// every slice product sum is an integer below 2^23, exact in fp32, and only
// the final combination is rounded (binary64).
#include <algorithm>
#include <cmath>
#include <mutex>

#include <cuda_fp16.h>

#include "block_codec.cuh"
#include "const_upload.cuh"
#include "gmap.cuh"

namespace blaz {

constexpr int kDotThreads = 256;

// Fixed-order CTA sum (warp shuffle tree, then the per-warp sums in order).
__device__ __forceinline__ double cta_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r += red[q];
    __syncthreads();
    return r;  // valid in thread 0
}

// Fixed-point slices of w and H (computed once on the host in long double).
constexpr int kSlices = 5;
struct GramConsts {
    float H[kSlices][kKeep][kKeep];  // integer digits, |digit| <= 2^10
    float w[kSlices][kKeep];
    double scaleH[kSlices], scaleW[kSlices];
    double inv_phi[256];             // 1/phi
};


// Tensor-core form of the Gram dot, 16 blocks per warp group.  Per slice s:
// Y_s = C_b H_s on mma.sync m16n8k16 with fp16 digits of H_s (|digit| <=
// 2^10, exact in fp16) and fp16 codes, every product sum an integer below
// 2^22, exact in the fp32 accumulators; w_s.c_b and w_s.c_a on two more
// products whose B operand holds w_s in every even column, so that every
// lane of a row's quad receives both rows' values; and sum_k c_a[k] Y_s[k]
// on the integer pipe: adding 1.5 2^23 to an accumulator makes its bits
// 0x4B400000 + Y_s[k], and 64-bit multiply-adds accumulate c_a[k] times those
// bits over the slices in Horner form (slices 0-2 and 3-4 in two
// accumulators).  The constant the offset contributes is taken off once,
// and the four lanes of a quad are summed once per group, not per slice.
struct GramTC {
    uint2 bfrag[kSlices][2][4][32];  // [slice][k-step][n-tile][lane]: H_s (columns 0..27)
    uint2 wfrag[kSlices][2][32];     // [slice][k-step][lane]: w_s in the even columns of one n-tile
    int eH2, eH4, eW2, eW4;          // log2 of scaleH[2], scaleH[4], scaleW[2], scaleW[4]
    double inv_phi[256];
};
__device__ GramTC g_gram;  // gram_tc(), copied once per device

// v 2^e as binary64 on the integer pipe (v's low bits beyond 53 truncated);
// e keeps the result a normal number for |v| < 2^63 (the slice scales).
__device__ __forceinline__ double i64_ldexp(long long v, int e)
{
    if (v == 0) return 0.0;
    const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const int msb = 63 - __clzll((long long)a);
    const unsigned long long m = msb <= 52 ? (a << (52 - msb)) : (a >> (msb - 52));
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(msb + e + 1023) << 52) | (m & 0x000FFFFFFFFFFFFFull)));
}

// 64 x on the exponent for normal x well inside the range, else a product.
__device__ __forceinline__ double times64(double x)
{
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    return (e >= 1 && e <= 2040) ? __longlong_as_double(b + (6ll << 52)) : 64.0 * x;
}

__device__ __forceinline__ void mma_f16x(float (&c)[4], const uint32_t (&a)[4], uint2 b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// The conversions below stay off the conversion unit (a quarter-rate pipe
// that the codes would otherwise saturate): a byte x ^ 0x80 = x + 128 placed
// under the exponent of 1024 (fp16) or 1.5 2^23 (fp32) is the number
// 1152 + x or 12583040 + x, and one exact subtraction leaves x.

// Two consecutive raw int8 codes (k, k+1) of a block, as 16 bits; zero beyond 28.
__device__ __forceinline__ uint32_t code_pair_raw(const int8_t *__restrict__ c, int k, bool valid)
{
    if (!valid || k >= kKeep) return 0u;
    return __ldg(reinterpret_cast<const uint16_t *>(c + k));
}

// A raw code pair as an fp16 pair (exact).
__device__ __forceinline__ uint32_t pair_to_h2(uint32_t v)
{
    const uint32_t q = __byte_perm(v ^ 0x8080u, 0x64646464u, 0x4140);
    const __half2 h = __hsub2(*reinterpret_cast<const __half2 *>(&q), __half2half2(__ushort_as_half((unsigned short)0x6480)));
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ uint32_t code_pair_h(const int8_t *__restrict__ c, int k, bool valid)
{
    return pair_to_h2(code_pair_raw(c, k, valid));
}

// One group of 16 blocks (rows gq and gq + 8 of the fragments).  On return
// every lane of a quad holds, for the row `row` it keeps (when `keep`), Q in
// two parts (qhi: slices 0-2 in units of slice 2, qlo: slices 3-4 in units of
// slice 4) and the per-slice values of w_s.c_a and w_s.c_b.
__device__ __forceinline__ void gram_group(const uint2 (*sbf)[2][4][32], const uint2 (*swf)[2][32], int64_t grp,
                                           int64_t nb, const int8_t *__restrict__ ca, const int8_t *__restrict__ cb,
                                           int lane, int gq, int t, int row, bool keep, long long &qhi,
                                           long long &qlo, float (&was)[kSlices], float (&wbs)[kSlices])
{
    const int64_t bA = grp * 16 + gq, bB = bA + 8;
    const bool vA = bA < nb, vB = bB < nb;
    const int8_t *cbA = cb + bA * kKeep, *cbB = cb + bB * kKeep;
    const int8_t *caA = ca + bA * kKeep, *caB = ca + bB * kKeep;
    // A fragments of the codes of both operands (k-steps 0 and 1)
    uint32_t b0[4], b1[4], a0[4], a1[4];
    b0[0] = code_pair_h(cbA, 2 * t, vA);
    b0[1] = code_pair_h(cbB, 2 * t, vB);
    b0[2] = code_pair_h(cbA, 2 * t + 8, vA);
    b0[3] = code_pair_h(cbB, 2 * t + 8, vB);
    b1[0] = code_pair_h(cbA, 16 + 2 * t, vA);
    b1[1] = code_pair_h(cbB, 16 + 2 * t, vB);
    b1[2] = code_pair_h(cbA, 24 + 2 * t, vA);
    b1[3] = code_pair_h(cbB, 24 + 2 * t, vB);
    // c_a at the 8 code positions this lane holds (k = nt*8 + 2t + {0,1}),
    // rows gq and gq + 8: raw pairs, their fp16 fragments and the integers
    uint32_t pA[4], pB[4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        pA[nt] = code_pair_raw(caA, nt * 8 + 2 * t, vA);
        pB[nt] = code_pair_raw(caB, nt * 8 + 2 * t, vB);
    }
    a0[0] = pair_to_h2(pA[0]);
    a0[1] = pair_to_h2(pB[0]);
    a0[2] = pair_to_h2(pA[1]);
    a0[3] = pair_to_h2(pB[1]);
    a1[0] = pair_to_h2(pA[2]);
    a1[1] = pair_to_h2(pB[2]);
    a1[2] = pair_to_h2(pA[3]);
    a1[3] = pair_to_h2(pB[3]);
    int xA[4][2], xB[4][2];
    int sA = 0, sB = 0;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            xA[nt][q] = (int)(int8_t)(uint8_t)(pA[nt] >> (8 * q));
            xB[nt][q] = (int)(int8_t)(uint8_t)(pB[nt] >> (8 * q));
            sA += xA[nt][q];
            sB += xB[nt][q];
        }
    long long hA = 0, lA = 0, hB = 0, lB = 0;
    const float2 magic = make_float2(12582912.0f, 12582912.0f);
#pragma unroll
    for (int sl = 0; sl < kSlices; ++sl) {
        long long &accA = sl < 3 ? hA : lA, &accB = sl < 3 ? hB : lB;
        if (sl != 0 && sl != 3) {
            accA *= 2048;
            accB *= 2048;
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma_f16x(c, b0, sbf[sl][0][nt][lane]);
            mma_f16x(c, b1, sbf[sl][1][nt][lane]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float2 y = __fadd2_rn(make_float2(c[q], c[2 + q]), magic);
                accA += (long long)xA[nt][q] * __float_as_int(y.x);
                accB += (long long)xB[nt][q] * __float_as_int(y.y);
            }
        }
        float d[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
        mma_f16x(d, b0, swf[sl][0][lane]);
        mma_f16x(d, b1, swf[sl][1][lane]);
        mma_f16x(e, a0, swf[sl][0][lane]);
        mma_f16x(e, a1, swf[sl][1][lane]);
        if (keep) {
            wbs[sl] = row ? d[2] : d[0];
            was[sl] = row ? e[2] : e[0];
        }
    }
    // the offset: sum_k c_a[k] 0x4B400000 per slice, times the Horner weights
    // (|sum| < 2^63 before and after: per slice and lane below 2^40.2)
    constexpr long long kOffHi = 0x4B400000ll * ((1ll << 22) + (1ll << 11) + 1);
    constexpr long long kOffLo = 0x4B400000ll * ((1ll << 11) + 1);
    hA -= kOffHi * sA;
    lA -= kOffLo * sA;
    hB -= kOffHi * sB;
    lB -= kOffLo * sB;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        hA += __shfl_xor_sync(0xffffffffu, hA, o);
        lA += __shfl_xor_sync(0xffffffffu, lA, o);
        hB += __shfl_xor_sync(0xffffffffu, hB, o);
        lB += __shfl_xor_sync(0xffffffffu, lB, o);
    }
    if (keep) {
        qhi = row ? hB : hA;
        qlo = row ? lB : lA;
    }
}

// Two groups of 16 blocks per warp step: lanes t = 0, 1 keep the sums of
// rows gq and gq + 8 of the first group, lanes t = 2, 3 those of the second,
// so the binary64 tail runs on all 32 lanes, one block each.
__global__ void __launch_bounds__(kDotThreads, 3)
    k_dot_tc(int64_t nb, const double *__restrict__ fa, const double *__restrict__ sa,
             const uint8_t *__restrict__ pa, const int8_t *__restrict__ ca, const double *__restrict__ fb,
             const double *__restrict__ sb, const uint8_t *__restrict__ pb, const int8_t *__restrict__ cb,
             double *__restrict__ partials, unsigned *__restrict__ counter, double *__restrict__ result,
             int64_t nbc, int64_t rows, int64_t cols, bool padded)
{
    __shared__ uint2 sbf[kSlices][2][4][32];
    __shared__ uint2 swf[kSlices][2][32];
    __shared__ double inv_phi[256];
    __shared__ double red[kDotThreads / 32];
    __shared__ bool last;
    const GramTC &g = g_gram;
    for (int i = threadIdx.x; i < kSlices * 2 * 4 * 32; i += blockDim.x) (&sbf[0][0][0][0])[i] = (&g.bfrag[0][0][0][0])[i];
    for (int i = threadIdx.x; i < kSlices * 2 * 32; i += blockDim.x) (&swf[0][0][0])[i] = (&g.wfrag[0][0][0])[i];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) inv_phi[i] = g.inv_phi[i];
    const int eH2 = g.eH2, eH4 = g.eH4, eW2 = g.eW2, eW4 = g.eW4;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
    const int wpc = blockDim.x >> 5;
    const int64_t npairs = (nb + 31) / 32;
    double acc1 = 0.0, acc2 = 0.0;
    for (int64_t pr = (int64_t)blockIdx.x * wpc + warp; pr < npairs; pr += (int64_t)gridDim.x * wpc) {
        long long qhi = 0, qlo = 0;
        float was[kSlices], wbs[kSlices];
#pragma unroll 1
        for (int half = 0; half < 2; ++half)  // not unrolled: one group's registers at a time
            gram_group(sbf, swf, 2 * pr + half, nb, ca, cb, lane, gq, t, t & 1, (t >> 1) == half, qhi, qlo, was,
                       wbs);
        // This lane's block: group 2 pr + (t >> 1), row gq + 8 (t & 1).
        const int64_t b = (2 * pr + (t >> 1)) * 16 + gq + 8 * (t & 1);
        bool use = b < nb;
        if (use && padded) {  // partial blocks of a padded matrix are left to k_dot_boundary
            const int64_t bi = b / nbc, bj = b - bi * nbc;
            use = bi * 8 + 8 <= rows && bj * 8 + 8 <= cols;
        }
        if (use) {
            // w slices assembled in int64 (0-2 and 3-4), then
            // fa (64 fb + tb Wb) + ta (fb Wa + tb Q)
            long long ahi = 0, alo = 0, bhi = 0, blo = 0;
#pragma unroll
            for (int sl = 0; sl < kSlices; ++sl) {
                const long long A = f2i_small(was[sl]), Bw = f2i_small(wbs[sl]);
                if (sl < 3) {
                    ahi = ahi * 2048 + A;
                    bhi = bhi * 2048 + Bw;
                } else {
                    alo = alo * 2048 + A;
                    blo = blo * 2048 + Bw;
                }
            }
            // ten binary64 operations: the power-of-two slice scales and the
            // factor 64 go to the exponent on the integer pipe
            const double Q = i64_ldexp(qhi, eH2) + i64_ldexp(qlo, eH4);
            const double Wa = i64_ldexp(ahi, eW2) + i64_ldexp(alo, eW4);
            const double Wb = i64_ldexp(bhi, eW2) + i64_ldexp(blo, eW4);
            const double ta = sa[b] * inv_phi[pa[b]], tb = sb[b] * inv_phi[pb[b]];
            const double f_a = fa[b], f_b = fb[b];
            const double t1 = fma(tb, Wb, times64(f_b));
            const double t2 = fma(tb, Q, f_b * Wa);
            acc1 = fma(f_a, t1, acc1);
            acc2 = fma(ta, t2, acc2);
        }
    }
    const double tot = cta_sum(acc1 + acc2, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = tot;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) v += __ldcg(partials + q);
    const double r = cta_sum(v, red);
    if (threadIdx.x == 0) {
        *result = r;
        *counter = 0u;
    }
}

// Host: G, w = G^T 1, H = G^T G in long double from the definitions, then the
// fixed-point slices.
static void slice(const long double *x, int n, float (*digits)[kKeep * kKeep], double *scale, int stride)
{
    long double mx = 0.0L;
    for (int i = 0; i < n; ++i) mx = std::max(mx, fabsl(x[i]));
    const int E = (mx > 0.0L ? (int)ceill(log2l(mx)) : 0) - 10;  // |x| / 2^E <= 2^10
    long double r[kKeep * kKeep];
    for (int i = 0; i < n; ++i) r[i] = x[i];
    for (int s = 0; s < kSlices; ++s) {
        const long double sc = ldexpl(1.0L, E - 11 * s);
        for (int i = 0; i < n; ++i) {
            const long double d = rintl(r[i] / sc);
            digits[s][i * stride / stride] = (float)d;
            r[i] -= d * sc;
        }
        scale[s] = (double)sc;
    }
}

static const GramConsts &gram_consts()
{
    static GramConsts g;
    static std::once_flag once;
    std::call_once(once, [] {
        const long double(*G)[kKeep] = decompress_map();
        long double H[kKeep * kKeep], w[kKeep];
        for (int k = 0; k < kKeep; ++k) {
            w[k] = 0.0L;
            for (int p = 0; p < 64; ++p) w[k] += G[p][k];
            for (int l = 0; l < kKeep; ++l) {
                long double acc = 0.0L;
                for (int p = 0; p < 64; ++p) acc += G[p][k] * G[p][l];
                H[k * kKeep + l] = acc;
            }
        }
        float hd[kSlices][kKeep * kKeep], wd[kSlices][kKeep * kKeep];
        slice(H, kKeep * kKeep, hd, g.scaleH, 1);
        slice(w, kKeep, wd, g.scaleW, 1);
        for (int s = 0; s < kSlices; ++s) {
            for (int k = 0; k < kKeep; ++k) {
                g.w[s][k] = wd[s][k];
                for (int l = 0; l < kKeep; ++l) g.H[s][k][l] = hd[s][k * kKeep + l];
            }
        }
        g.inv_phi[0] = 0.0;
        for (int p = 1; p < 256; ++p) g.inv_phi[p] = 1.0 / (double)p;
    });
    return g;
}

// Algorithm 3 generalised to matrices.  Line ri of block (bi, kb) of A is
// fa + ta G_r ca (G_r: rows 8 ri .. 8 ri + 7 of the decompression map) and
// column cj of block (kb, bj) of B is fb + tb G_c cb (rows cj, cj + 8, ...),
// so only the needed line and column are decompressed (IPREDICT_LINES /
// IPREDICT_COLS of Algorithm 3).  16 lanes per k-block; CTA partials are
// added in order by the last CTA.
struct RowColConsts {
    double G[64][kKeep];
    double inv_phi[256];
};
__device__ RowColConsts g_rowcol;  // rowcol_consts(), copied once per device

__global__ void __launch_bounds__(kDotThreads)
    k_dot_rowcol(int64_t nkb, int64_t nbc_a, int64_t nbc_b, int64_t i,
                 int64_t j, const double *__restrict__ fa, const double *__restrict__ sa,
                 const uint8_t *__restrict__ pa, const int8_t *__restrict__ ca, const double *__restrict__ fb,
                 const double *__restrict__ sb, const uint8_t *__restrict__ pb, const int8_t *__restrict__ cb,
                 double *__restrict__ partials, unsigned *__restrict__ counter, double *__restrict__ result)
{
    __shared__ double red[kDotThreads / 32];
    __shared__ bool last;
    // the 8 rows of G for line ri, the 8 for column cj, and 1/phi (shared:
    // uniform reads broadcast, per-lane reads of 1/phi spread over banks)
    __shared__ double Gr[8][kKeep], Gc[8][kKeep], inv_phi[256];
    const int64_t bi = i / 8, bj = j / 8;
    const int ri = (int)(i % 8), cj = (int)(j % 8);
    for (int e = threadIdx.x; e < 8 * kKeep; e += blockDim.x) {
        const int q = e / kKeep, t = e - q * kKeep;
        Gr[q][t] = g_rowcol.G[ri * 8 + q][t];
        Gc[q][t] = g_rowcol.G[q * 8 + cj][t];
    }
    for (int e = threadIdx.x; e < 256; e += blockDim.x) inv_phi[e] = g_rowcol.inv_phi[e];
    __syncthreads();
    // A team of 16 lanes per k-block: lane (side, q) decodes entry q of the
    // line (side 0, block (bi, kb)) or of the column (side 1, block (kb, bj))
    // with one row of G, so the binary64 chains of a block are spread over
    // 16 lanes (a warp's binary64 instruction costs the same for 1 lane as
    // for 32, and one warp per SM sub-partition issues few of them).
    const int lane = threadIdx.x & 31, side = (lane >> 3) & 1, q = lane & 7;
    const unsigned tmask = 0xFFFFu << (lane & 16);
    const double *Gq = side ? Gc[q] : Gr[q];
    double acc = 0.0;
    const int64_t teams = (int64_t)gridDim.x * blockDim.x / 16;
    for (int64_t kb = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 16; kb < nkb; kb += teams) {
        const int64_t b = side ? kb * nbc_b + bj : bi * nbc_a + kb;
        int8_t x[kKeep];
        load_codes((side ? cb : ca) + b * kKeep, x);
        double y = 0.0;
#pragma unroll
        for (int t = 0; t < kKeep; ++t) y = fma(Gq[t], i64_to_double(x[t]), y);
        const double v = fma((side ? sb[b] : sa[b]) * inv_phi[side ? pb[b] : pa[b]], y, side ? fb[b] : fa[b]);
        const double w = __shfl_xor_sync(tmask, v, 8);
        double prod = side ? 0.0 : v * w;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) prod += __shfl_xor_sync(tmask, prod, o);
        if ((lane & 15) == 0) acc += prod;
    }
    const double tot = cta_sum(acc, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = tot;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) v += __ldcg(partials + q);
    const double r = cta_sum(v, red);
    if (threadIdx.x == 0) {
        *result = r;
        *counter = 0u;
    }
}

static const RowColConsts &rowcol_consts()
{
    static RowColConsts g;
    static std::once_flag once;
    std::call_once(once, [] {
        const long double(*G)[kKeep] = decompress_map();
        for (int p = 0; p < 64; ++p)
            for (int t = 0; t < kKeep; ++t) g.G[p][t] = (double)G[p][t];
        g.inv_phi[0] = 0.0;
        for (int p = 1; p < 256; ++p) g.inv_phi[p] = 1.0 / (double)p;
    });
    return g;
}

static const GramTC &gram_tc()
{
    static GramTC tcc;
    static std::once_flag once;
    std::call_once(once, [] {
        const GramConsts &gc = gram_consts();
        auto h2 = [](float lo, float hi) {
            const __half a = __float2half_rn(lo), b = __float2half_rn(hi);
            return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
        };
        // B[k = l (code of cb)][n] = H_s[n][l] for n, l < 28, else 0.
        auto bval = [&](int s, int l, int n) -> float { return l < kKeep && n < kKeep ? gc.H[s][n][l] : 0.0f; };
        // B[k = l][n] = w_s[l] in the even columns n of the w product.
        auto wval = [&](int s, int l, int n) -> float { return l < kKeep && n % 2 == 0 ? gc.w[s][l] : 0.0f; };
        for (int s = 0; s < kSlices; ++s)
            for (int ks = 0; ks < 2; ++ks)
                for (int lane = 0; lane < 32; ++lane) {
                    const int gg = lane >> 2, t = lane & 3, k = ks * 16 + 2 * t;
                    for (int nt = 0; nt < 4; ++nt) {
                        const int n = nt * 8 + gg;
                        tcc.bfrag[s][ks][nt][lane].x = h2(bval(s, k, n), bval(s, k + 1, n));
                        tcc.bfrag[s][ks][nt][lane].y = h2(bval(s, k + 8, n), bval(s, k + 9, n));
                    }
                    tcc.wfrag[s][ks][lane].x = h2(wval(s, k, gg), wval(s, k + 1, gg));
                    tcc.wfrag[s][ks][lane].y = h2(wval(s, k + 8, gg), wval(s, k + 9, gg));
                }
        tcc.eH2 = std::ilogb(gc.scaleH[2]);
        tcc.eH4 = std::ilogb(gc.scaleH[4]);
        tcc.eW2 = std::ilogb(gc.scaleW[2]);
        tcc.eW4 = std::ilogb(gc.scaleW[4]);
        for (int p = 0; p < 256; ++p) tcc.inv_phi[p] = gc.inv_phi[p];
    });
    return tcc;
}

int dot_grid(int64_t nb)
{
    int64_t want = ((nb + 31) / 32 + (kDotThreads / 32) - 1) / (kDotThreads / 32);  // 32 blocks per warp step
    // two resident waves (3 CTAs of 256 threads per SM), never more than the
    // kDotMaxCtas partial sums of the no-allocation entry point
    int64_t cap = std::min<int64_t>((int64_t)num_sms() * 6, kDotMaxCtas);
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

// The partial blocks of a padded matrix pair (the last block row when rows is
// not a multiple of 8, then the last block column when cols is not, without
// the corner twice): each thread decompresses one block of each operand in
// binary64 and sums the products of its logical entries, row-major.  CTA
// partials are added in CTA order by the last CTA, which adds the sum of the
// full blocks already in *result.
__global__ void __launch_bounds__(kDotThreads)
    k_dot_boundary(const double *__restrict__ fa, const double *__restrict__ sa, const uint8_t *__restrict__ pa,
                   const int8_t *__restrict__ ca, const double *__restrict__ fb, const double *__restrict__ sb,
                   const uint8_t *__restrict__ pb, const int8_t *__restrict__ cb, int64_t nbr, int64_t nbc,
                   int64_t rows, int64_t cols, int64_t nbd, double *__restrict__ partials,
                   unsigned *__restrict__ counter, double *__restrict__ result)
{
    __shared__ double red[kDotThreads / 32];
    __shared__ bool last;
    const int64_t nrow = rows % 8 ? nbc : 0;
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nbd; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bi = q < nrow ? nbr - 1 : q - nrow, bj = q < nrow ? q : nbc - 1;
        const int64_t b = bi * nbc + bj;
        double x[64], y[64];
        decompress_block_at(fa[b], sa[b], pa[b], ca + b * kKeep, x);
        decompress_block_at(fb[b], sb[b], pb[b], cb + b * kKeep, y);
        const int64_t ri = rows - bi * 8 < 8 ? rows - bi * 8 : 8, cj = cols - bj * 8 < 8 ? cols - bj * 8 : 8;
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (i < ri && j < cj) acc = fma(x[i * 8 + j], y[i * 8 + j], acc);
    }
    const double tot = cta_sum(acc, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = tot;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) v += __ldcg(partials + q);
    const double r = cta_sum(v, red);
    if (threadIdx.x == 0) {
        *result = __ldcg(result) + r;
        *counter = 0u;
    }
}

int launch_dot(const blaz_cmat *a, const blaz_cmat *b, double *result, double *partials, unsigned *counter,
               int64_t max_ctas, cudaStream_t st, int64_t rows, int64_t cols)
{
    const int64_t nbc = a->cols / 8, nb = (a->rows / 8) * nbc;
    if (rows < 0) rows = a->rows;
    if (cols < 0) cols = a->cols;
    const bool padded = rows != a->rows || cols != a->cols;
    int grid = dot_grid(nb);
    if (grid > max_ctas) grid = (int)max_ctas;
    static DeviceTable table;
    int rc = table.ensure(&g_gram, &gram_tc(), sizeof(GramTC), 0, st);
    if (rc) return rc;
    k_dot_tc<<<grid, kDotThreads, 0, st>>>(nb, a->f, a->s, a->phi, a->code, b->f, b->s, b->phi,
                                           b->code, partials, counter, result, nbc, rows, cols, padded);
    rc = launch_status();
    if (rc || !padded) return rc;
    // The partial blocks: the last block row and/or the last block column.
    const int64_t nbr = a->rows / 8;
    const int64_t nbd = (rows % 8 ? nbc : 0) + (cols % 8 ? nbr - (rows % 8 ? 1 : 0) : 0);
    // One warp per CTA: each thread decodes two blocks in binary64, so the
    // O(n) partial blocks are spread over as many SMs as possible.
    const int64_t want = (nbd + 31) / 32;
    const int bgrid = (int)std::max<int64_t>(1, std::min<int64_t>(want, max_ctas));
    k_dot_boundary<<<bgrid, 32, 0, st>>>(a->f, a->s, a->phi, a->code, b->f, b->s, b->phi, b->code, nbr,
                                                  nbc, rows, cols, nbd, partials, counter, result);
    return launch_status();
}

int rowcol_grid(int64_t nkb)
{
    int64_t want = (nkb * 16 + kDotThreads - 1) / kDotThreads;
    const int64_t cap = (int64_t)num_sms();
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

int launch_dot_rowcol(const blaz_cmat *a, const blaz_cmat *b, int64_t i, int64_t j, double *result,
                      double *partials, unsigned *counter, cudaStream_t st)
{
    const int64_t nkb = a->cols / 8;
    const int grid = rowcol_grid(nkb);
    static DeviceTable table;
    const int rc = table.ensure(&g_rowcol, &rowcol_consts(), sizeof(RowColConsts), 0, st);
    if (rc) return rc;
    k_dot_rowcol<<<grid, kDotThreads, 0, st>>>(nkb, a->cols / 8, b->cols / 8, i, j, a->f, a->s,
                                               a->phi, a->code, b->f, b->s, b->phi, b->code, partials, counter,
                                               result);
    return launch_status();
}

}  // namespace blaz
