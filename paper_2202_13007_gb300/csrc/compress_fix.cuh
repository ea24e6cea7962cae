// compress_fix.cuh -- the exact binary64 evaluation, by a team of 8 lanes,
// of the blocks and codes the certified compressor (compress_fast.cuh) could
// not decide; shared by the two-kernel compressor and the batch kernel.
// Compression of Sec. II of "Compressed Matrix Computations" (arXiv
// 2202.13007), in the binary64 operation order of include/blaz.h.
#pragma once

#include "compress_fast.cuh"

namespace blaz {

// Row u of D for block b, exactly as compress_block forms it: Eq. eqnorm
// from rows u and u-1 of the input.  Rows and columns beyond the logical
// rows x cols repeat the last one (padding).
__device__ __forceinline__ void team_d_row(const double *__restrict__ A, int64_t lda, int64_t rows, int64_t cols,
                                           int64_t nbc, int64_t b, int u, double (&dp)[8])
{
    const int64_t bi = b / nbc, bj = b - (b / nbc) * nbc;
    const int64_t r = bi * 8 + u < rows ? bi * 8 + u : rows - 1;
    const int64_t rp = bi * 8 + u - 1 < rows ? bi * 8 + u - 1 : rows - 1;
    double cur[8], prev[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const int64_t c = bj * 8 + v < cols ? bj * 8 + v : cols - 1;
        cur[v] = __ldg(A + r * lda + c);
        prev[v] = u > 0 ? __ldg(A + rp * lda + c) : 0.0;
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if (u == 0) dp[v] = v == 0 ? 0.0 : dsub(cur[v], cur[v - 1]);
        else if (v == 0) dp[v] = dsub(cur[0], prev[0]);
        else dp[v] = dhalf(dadd(dsub(cur[v], prev[v]), dsub(cur[v], cur[v - 1])));
    }
}

// Row u of D' = D times r = 1/s (s as stored).
template <bool kVec>
__device__ __forceinline__ void team_dprime_row(const double *__restrict__ A, int64_t lda, int64_t rows, int64_t cols,
                                                int64_t nbc, int64_t b, int u, double s, double (&dp)[8])
{
    team_d_row(A, lda, rows, cols, nbc, b, u, dp);
    const double rs = ddiv(1.0, s);
#pragma unroll
    for (int v = 0; v < 8; ++v) dp[v] = dmul(dp[v], rs);
}

// Whole blocks whose phi was not certified (or with non-finite values): the
// exact binary64 compressor by the team of 8 lanes.  s is already exact
// (k_compress_fast stores it for every block).  Lane u forms row u of D' and
// the inner sums T_j[u] of all eight columns; lane i then forms
// U[i][j] = sum_u cos_iu T_j[u] in the specified order from the team's
// shuffles, X[i][j], and its share of m = max |X| (NaN ignored, as in
// compress_block: the maximum of non-NaN values is order-free).
template <bool kVec>
__device__ __forceinline__ void fix_whole_block(const double *__restrict__ A, int64_t lda, int64_t rows, int64_t cols,
                                                int64_t nbc, int64_t b,
                                                const double *__restrict__ s, uint8_t *__restrict__ phi,
                                                int8_t *__restrict__ code, int u, int tbase, unsigned tmask)
{
    double ci[8];  // cos_{u,x}: this lane's row of the cosine table as output row i = u
#pragma unroll
    for (int x = 0; x < 8; ++x) ci[x] = c_cos[u * 8 + x];
    double dp[8];
    team_dprime_row<kVec>(A, lda, rows, cols, nbc, b, u, s[b], dp);
    double T[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        double acc = (j == 0) ? dp[0] : dmul(dp[0], cos_tab(j, 0));
#pragma unroll
        for (int v = 1; v < 8; ++v) acc = dadd(acc, (j == 0) ? dp[v] : dmul(dp[v], cos_tab(j, v)));
        T[j] = acc;
    }
    double U[8];
#pragma unroll
    for (int uu = 0; uu < 8; ++uu) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const double Tu = __shfl_sync(tmask, T[j], tbase + uu);
            const double term = (u == 0) ? Tu : dmul(ci[uu], Tu);
            U[j] = (uu == 0) ? term : dadd(U[j], term);
        }
    }
    double m = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        U[j] = dmul((u == 0 && j == 0) ? BLAZ_A00 : (u == 0 || j == 0) ? BLAZ_A0K : BLAZ_AKK, U[j]);
        const double ax = fabs(U[j]);
        m = (ax > m) ? ax : m;
    }
#pragma unroll
    for (int off = 4; off; off >>= 1) {
        const double o = __shfl_xor_sync(tmask, m, off);
        m = (o > m) ? o : m;
    }
    const int ph = phi_of(m);
    const double phd = i64_to_double(ph);
    if (u == 0) phi[b] = (uint8_t)ph;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int t = kept_index(u, j);
        if (t >= 0) code[b * kKeep + t] = quantize_bits(dmul(U[j], phd));
    }
}

// Undecided codes of block b (bit t of `pending` for code t), phi already
// set: for each, the team forms the inner sums T[u] (lane u) and the outer
// sum over u in the specified order from the shuffles.
template <bool kVec>
__device__ __forceinline__ void fix_codes_of_block(const double *__restrict__ A, int64_t lda, int64_t rows,
                                                   int64_t cols, int64_t nbc, int64_t b,
                                                   uint32_t pending, const double *__restrict__ s,
                                                   const uint8_t *__restrict__ phi, int8_t *__restrict__ code, int u,
                                                   int tbase, unsigned tmask)
{
    double dp[8];
    team_dprime_row<kVec>(A, lda, rows, cols, nbc, b, u, s[b], dp);
    const int ph = phi[b];
    for (uint32_t m = pending; m; m &= m - 1) {
        const int t = __ffs(m) - 1;
        const int i = kept_row(t), j = kept_col(t);
        double T = (j == 0) ? dp[0] : dmul(dp[0], c_cos[j * 8]);
#pragma unroll
        for (int v = 1; v < 8; ++v) T = dadd(T, (j == 0) ? dp[v] : dmul(dp[v], c_cos[j * 8 + v]));
        double U = 0.0;
#pragma unroll
        for (int uu = 0; uu < 8; ++uu) {
            const double Tu = __shfl_sync(tmask, T, tbase + uu);
            const double term = (i == 0) ? Tu : dmul(c_cos[i * 8 + uu], Tu);
            U = (uu == 0) ? term : dadd(U, term);
        }
        if (u == 0) {
            const double aa = (i == 0 && j == 0) ? BLAZ_A00 : (i == 0 || j == 0) ? BLAZ_A0K : BLAZ_AKK;
            code[b * kKeep + t] = quantize_bits(dmul(dmul(aa, U), i64_to_double(ph)));
        }
    }
}

// Undecided codes of block b (bit t of `pending`: code t) by one lane, phi
// already set: the block's D by the integer form of Eq. eqnorm when the
// block is uniform (else on the binary64 pipe), D' = D (1/s) with s as
// stored, and each listed code in the specified order,
//     T_u = sum_v D'_uv cos_jv (v ascending),  U = sum_u cos_iu T_u (u ascending),
//     code = quantize(RN(aa_ij U) phi),
// where products by cos 0 = 1 are exact (same bits as omitting them).
// cs: the cosine table in shared memory (the lanes of a warp evaluate
// different codes).  One lane per block costs a quarter of the binary64
// warp instructions of a team of 8 lanes for the usual single code.
template <bool kVec>
__device__ __forceinline__ void fix_codes_lane(const double *__restrict__ A, int64_t lda, int64_t rows, int64_t cols,
                                               int64_t nbc, int64_t b, uint32_t pending,
                                               const double *__restrict__ s, const uint8_t *__restrict__ phi,
                                               int8_t *__restrict__ code, const double *cs)
{
    double d[64];
    const int64_t bi = b / nbc, bj = b - bi * nbc;
    if (bi * 8 + 8 <= rows && bj * 8 + 8 <= cols) load_block<kVec>(A, lda, bi, bj, d);
    else load_block_clamped(A, lda, bi, bj, rows, cols, d);
    if (block_is_uniform(d)) {
        const unsigned hi0 = (unsigned)__double2hiint(d[0]);
        const int e = (int)((hi0 >> 20) & 0x7FFu);
        int K;
        unsigned pos, neg;
        normalize_uniform(d, e, hi0 >> 31, K, pos, neg);
#pragma unroll
        for (int p = 0; p < 64; ++p) d[p] = uniform_d(__double_as_longlong(d[p]), e, hi0 >> 31);
    } else {
        normalize_block(d);
    }
    const double r = ddiv(1.0, s[b]);
#pragma unroll
    for (int p = 0; p < 64; ++p) d[p] = dmul(d[p], r);
    const double phd = i64_to_double(phi[b]);
    for (uint32_t m = pending; m; m &= m - 1u) {
        const int t = __ffs(m) - 1, i = kept_row(t), j = kept_col(t);
        double cj[8], ci[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            cj[x] = cs[j * 8 + x];
            ci[x] = cs[i * 8 + x];
        }
        double U = 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            double T = dmul(d[u * 8], cj[0]);
#pragma unroll
            for (int v = 1; v < 8; ++v) T = dadd(T, dmul(d[u * 8 + v], cj[v]));
            const double term = dmul(ci[u], T);
            U = (u == 0) ? term : dadd(U, term);
        }
        const double aa = (i == 0 && j == 0) ? BLAZ_A00 : (i == 0 || j == 0) ? BLAZ_A0K : BLAZ_AKK;
        code[b * kKeep + t] = quantize_bits(dmul(dmul(aa, U), phd));
    }
}

}  // namespace blaz
