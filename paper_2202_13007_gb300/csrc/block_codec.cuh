// block_codec.cuh -- per-block device code shared by the standalone kernels
// and the persistent batch kernel: loading a block, compressing it (Sec. II of
// "Compressed Matrix Computations", arXiv 2202.13007; bit-exact binary64
// order fixed in include/blaz.h), code packing, and decompressing a block.
#pragma once

#include "blaz_internal.cuh"

namespace blaz {

// One thread per 8x8 block.  Loads the block (eight rows of 64 B) with 16-byte
// vector loads when the matrix allows it.
template <bool kVec>
__device__ __forceinline__ void load_block(const double *__restrict__ A, int64_t lda, int64_t bi, int64_t bj,
                                           double (&d)[64])
{
    const double *p = A + (bi * 8) * lda + bj * 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (kVec) {
            const double2 *q = reinterpret_cast<const double2 *>(p + i * lda);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                double2 v = __ldg(q + h);
                d[i * 8 + 2 * h] = v.x;
                d[i * 8 + 2 * h + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) d[i * 8 + j] = __ldg(p + i * lda + j);
        }
    }
}

// Block (bi, bj) of the edge-replicated extension of a rows x cols matrix
// (rows, cols >= 1): entry (r, c) reads A at (min(r, rows-1), min(c, cols-1)).
__device__ __forceinline__ void load_block_clamped(const double *__restrict__ A, int64_t lda, int64_t bi,
                                                   int64_t bj, int64_t rows, int64_t cols, double (&d)[64])
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = bi * 8 + i < rows ? bi * 8 + i : rows - 1;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t c = bj * 8 + j < cols ? bj * 8 + j : cols - 1;
            d[i * 8 + j] = __ldg(A + r * lda + c);
        }
    }
}

// Compress one block held in d (overwritten).  Writes s, phi and the 28 codes.
__device__ __forceinline__ void compress_block(double (&d)[64], double &s_out, uint8_t &phi_out,
                                               int8_t (&code)[kKeep])
{
    // Eq. eqnorm, evaluated in place from the last element backwards so that
    // M(i-1,j) and M(i,j-1) are still the inputs when D(i,j) is formed.
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
                double a = dsub(d[i * 8 + j], d[(i - 1) * 8 + j]);
                double b = dsub(d[i * 8 + j], d[i * 8 + j - 1]);
                d[i * 8 + j] = dmul(dadd(a, b), 0.5);
            }
        }
    }
    // Eqs. eqslope / eqslope2: K nonzero entries, S = sum |D| (pairwise tree).
    int K = 0;
#pragma unroll
    for (int p = 0; p < 64; ++p) K += (d[p] != 0.0);
    const double S = tree_sum_abs(d);
    if (K == 0) {  // constant block: s = 0, all coefficients 0, phi = 127/0 -> 255
        s_out = 0.0;
        phi_out = 255;
#pragma unroll
        for (int t = 0; t < kKeep; ++t) code[t] = 0;
        return;
    }
    const double s = ddiv(S, (double)K);
    const double r = ddiv(1.0, s);
#pragma unroll
    for (int p = 0; p < 64; ++p) d[p] = dmul(d[p], r);
    s_out = s;

    // Eq. eqdct, one output column j at a time: inner sums T[u] over v, outer
    // sums over u, then the alpha_i alpha_j factor.  Multiplications by
    // cos(0) = 1 are exact and therefore omitted.
    double kept[kKeep];
    double m = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        double T[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            double acc = (j == 0) ? d[u * 8] : dmul(d[u * 8], cos_tab(j, 0));
#pragma unroll
            for (int v = 1; v < 8; ++v) acc = dadd(acc, (j == 0) ? d[u * 8 + v] : dmul(d[u * 8 + v], cos_tab(j, v)));
            T[u] = acc;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            double acc = (i == 0) ? T[0] : dmul(cos_tab(i, 0), T[0]);
#pragma unroll
            for (int u = 1; u < 8; ++u) acc = dadd(acc, (i == 0) ? T[u] : dmul(cos_tab(i, u), T[u]));
            const double X = dmul(aa_tab(i, j), acc);
            const double ax = fabs(X);
            m = (ax > m) ? ax : m;
            const int t = kept_index(i, j);
            if (t >= 0) kept[t] = X;
        }
    }
    // Eq. eqphi
    const double q = ddiv(127.0, m);
    int phi;
    if (!(q < 255.0)) phi = 255;
    else {
        phi = __double2int_rz(q);
        phi = phi < 1 ? 1 : phi;
    }
    phi_out = (uint8_t)phi;
    const double phid = (double)phi;
#pragma unroll
    for (int t = 0; t < kKeep; ++t) code[t] = quantize(dmul(kept[t], phid));
}

__device__ __forceinline__ void store_codes(int8_t *__restrict__ dst, const int8_t (&code)[kKeep])
{
    // 28 bytes at a 4-byte aligned address (block * 28).
    uint32_t *w = reinterpret_cast<uint32_t *>(dst);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        uint32_t v = (uint32_t)(uint8_t)code[4 * q] | ((uint32_t)(uint8_t)code[4 * q + 1] << 8) |
                     ((uint32_t)(uint8_t)code[4 * q + 2] << 16) | ((uint32_t)(uint8_t)code[4 * q + 3] << 24);
        w[q] = v;
    }
}

__device__ __forceinline__ void load_codes(const int8_t *__restrict__ src, int8_t (&code)[kKeep])
{
    const uint32_t *w = reinterpret_cast<const uint32_t *>(src);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        uint32_t v = __ldg(w + q);
#pragma unroll
        for (int b = 0; b < 4; ++b) code[4 * q + b] = (int8_t)(uint8_t)(v >> (8 * b));
    }
}

// ---------------------------------------------------------------------------------
// Decompression of one block into registers: X = code/phi (kept positions),
// D_hat = s * IDCT(X), then the inverse of Eq. eqnorm.  Floating-point result
// compared within a tolerance; fused multiply-adds are used freely.
__device__ __forceinline__ void decompress_block(double f, double s, int phi, const int8_t (&code)[kKeep],
                                                 double (&out)[64])
{
    const double inv = 1.0 / (double)phi;
    // Y = alpha_i alpha_j * code / phi on the kept positions.
    double Y[kKeep];
#pragma unroll
    for (int t = 0; t < kKeep; ++t) Y[t] = aa_tab(kept_row(t), kept_col(t)) * ((double)code[t] * inv);
    // P = C^T Y C, computed one output column v at a time.
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        double Q[8];  // Q[i] = sum_j Y[i][j] cos_jv
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            double acc = Y[kept_index(i, 0)];
            acc = fma(Y[kept_index(i, 1)], cos_tab(1, v), acc);
            if (i < 2) {
#pragma unroll
                for (int j = 2; j < 8; ++j) acc = fma(Y[kept_index(i, j)], cos_tab(j, v), acc);
            }
            Q[i] = acc;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            double acc = Q[0];
#pragma unroll
            for (int i = 1; i < 8; ++i) acc = fma(cos_tab(i, u), Q[i], acc);
            out[u * 8 + v] = s * acc;  // D_hat(u, v)
        }
    }
    // inverse normalization (row-major order: every dependency is earlier)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            double v;
            if (i == 0 && j == 0) v = f;
            else if (i == 0) v = out[j - 1] + out[j];
            else if (j == 0) v = out[(i - 1) * 8] + out[i * 8];
            else v = fma(out[(i - 1) * 8 + j] + out[i * 8 + j - 1], 0.5, out[i * 8 + j]);
            out[i * 8 + j] = v;
        }
    }
}

__device__ __forceinline__ void decompress_block_at(double f, double s, int phi, const int8_t *__restrict__ code,
                                                    double (&out)[64])
{
    int8_t c[kKeep];
    load_codes(code, c);
    decompress_block(f, s, phi, c, out);
}

}  // namespace blaz
