// block_codec.cuh -- per-block device helpers shared by the kernels that read
// compressed blocks: code packing and the decompression of one block
// (inverse of Sec. II of "Compressed Matrix Computations", arXiv 2202.13007).
#pragma once

#include "blaz_internal.cuh"

namespace blaz {

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
