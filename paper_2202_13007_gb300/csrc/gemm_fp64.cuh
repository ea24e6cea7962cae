// gemm_fp64.cuh -- binary64 tile product on the FP64 tensor path of sm_103a
// (mma.sync.m8n8k4.f64, DMMA; tcgen05 has no f64 kind), shared by the
// standalone product kernel and the persistent batch kernel.  Used by the
// compressed matrix product ("Matrix multiplication", Sec. III of
// "Compressed Matrix Computations", arXiv 2202.13007).
#pragma once

#include "blaz_internal.cuh"

namespace blaz {

__device__ __forceinline__ void dmma_8x8x4(double (&c)[2], double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a), "d"(b));
}

constexpr int kGemmBM = 64, kGemmBN = 64, kGemmBK = 16;
constexpr int kGemmLdaS = kGemmBK + 4;  // padded strides: conflict-free fragment reads
constexpr int kGemmLdbS = kGemmBN + 4;
constexpr int kGemmThreads = 128;       // 4 warps, 2 x 2, each a 32 x 32 warp tile

struct GemmSmem {
    double As[2][kGemmBM][kGemmLdaS];
    double Bs[2][kGemmBK][kGemmLdbS];
};

// One 64 x 64 tile (rows row0.., columns col0..) of C = A * B, computed by
// the calling CTA of kGemmThreads threads with DMMA.  A is 16-byte aligned with
// even lda and n, k multiples of 8; any m >= 1.  With kCoherentA the A
// operand is read through L2 only (it may have been written earlier in the
// same kernel by other CTAs).
template <bool kCoherentA>
__device__ __forceinline__ void gemm_tile_fp64(GemmSmem &sm, const double *__restrict__ A, int64_t lda,
                                               const double *__restrict__ B, int64_t ldb, double *__restrict__ C,
                                               int64_t ldc, int64_t n, int64_t k, int64_t m, int64_t row0,
                                               int64_t col0)
{
    auto &As = sm.As;
    auto &Bs = sm.Bs;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;

    double acc[4][4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;

    // Global -> register staging: A: row tid/2, 8 columns; B: row tid/8, 8 columns.
    double ra[8], rb[8];
    const int ar = tid >> 1, ac = (tid & 1) * 8;
    const int br = tid >> 3, bc = (tid & 7) * 8;
    auto load = [&](int64_t k0) {
        const int64_t gr = row0 + ar;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double2 v = make_double2(0.0, 0.0);
            if (gr < n && k0 + ac + 2 * q < k) v = kCoherentA ? __ldcg(reinterpret_cast<const double2 *>(A + gr * lda + k0 + ac) + q)
                               : __ldg(reinterpret_cast<const double2 *>(A + gr * lda + k0 + ac) + q);
            ra[2 * q] = v.x;
            ra[2 * q + 1] = v.y;
        }
        const int64_t gk = k0 + br;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t gc = col0 + bc + q;
            rb[q] = (gk < k && gc < m) ? __ldg(B + gk * ldb + gc) : 0.0;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 8; ++q) As[buf][ar][ac + q] = ra[q];
#pragma unroll
        for (int q = 0; q < 8; ++q) Bs[buf][br][bc + q] = rb[q];
    };

    const int64_t ktiles = (k + kGemmBK - 1) / kGemmBK;
    load(0);
    store(0);
    __syncthreads();
    for (int64_t kt = 0; kt < ktiles; ++kt) {
        const int buf = (int)(kt & 1);
        if (kt + 1 < ktiles) load((kt + 1) * kGemmBK);
#pragma unroll
        for (int kk = 0; kk < kGemmBK; kk += 4) {
            double af[4], bf[4];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) af[mi] = As[buf][wm + mi * 8 + g][kk + t];
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) bf[ni] = Bs[buf][kk + t][wn + ni * 8 + g];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) dmma_8x8x4(acc[mi][ni], af[mi], bf[ni]);
        }
        if (kt + 1 < ktiles) store(buf ^ 1);
        __syncthreads();
    }
    // Epilogue: c0, c1 = C[g][2t], C[g][2t+1] of each 8 x 8 tile.
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const int64_t r = row0 + wm + mi * 8 + g;
            const int64_t c = col0 + wn + ni * 8 + 2 * t;
            if (r < n) {
                if (c < m) C[r * ldc + c] = acc[mi][ni][0];
                if (c + 1 < m) C[r * ldc + c + 1] = acc[mi][ni][1];
            }
        }
}


}  // namespace blaz
