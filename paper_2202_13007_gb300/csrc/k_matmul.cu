// k_matmul.cu -- dense products used by the compressed matrix product
// ("Matrix multiplication", Sec. III of "Compressed Matrix Computations",
// arXiv 2202.13007): the compressed operand is decompressed once into a
// stream-ordered scratch matrix, then multiplied here.
//
// FP64 path: mma.sync.m8n8k4.f64 (DMMA), the binary64 tensor instruction of
// sm_103a (tcgen05 has no f64 kind).
#include "blaz_internal.cuh"

namespace blaz {

namespace {
constexpr int BM = 64, BN = 64, BK = 16;
constexpr int LDA_S = BK + 4;  // padded strides: conflict-free fragment reads
constexpr int LDB_S = BN + 4;
constexpr int kThreads = 128;  // 4 warps, 2 x 2, each a 32 x 32 warp tile
}  // namespace

__device__ __forceinline__ void dmma_8x8x4(double (&c)[2], double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a), "d"(b));
}

// C (n x m) = A (n x k) * B (k x m); row-major; n, k multiples of 8; any m >= 1.
// A is 16-byte aligned with even lda (the decompressed scratch operand).
__global__ void __launch_bounds__(kThreads)
    k_gemm_fp64(const double *__restrict__ A, int64_t lda, const double *__restrict__ B, int64_t ldb,
                double *__restrict__ C, int64_t ldc, int64_t n, int64_t k, int64_t m)
{
    __shared__ double As[2][BM][LDA_S];
    __shared__ double Bs[2][BK][LDB_S];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int64_t row0 = (int64_t)blockIdx.y * BM, col0 = (int64_t)blockIdx.x * BN;

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
            if (gr < n && k0 + ac + 2 * q < k) v = __ldg(reinterpret_cast<const double2 *>(A + gr * lda + k0 + ac) + q);
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

    const int64_t ktiles = (k + BK - 1) / BK;
    load(0);
    store(0);
    __syncthreads();
    for (int64_t kt = 0; kt < ktiles; ++kt) {
        const int buf = (int)(kt & 1);
        if (kt + 1 < ktiles) load((kt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; kk += 4) {
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

int launch_gemm_fp64(const double *A, int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc, int64_t n,
                     int64_t k, int64_t m, cudaStream_t st)
{
    if (n == 0 || m == 0) return BLAZ_OK;
    if ((n + BM - 1) / BM > 65535 || (m + BN - 1) / BN > 0x7fffffff) return BLAZ_ERR_SHAPE;
    dim3 grid((unsigned)((m + BN - 1) / BN), (unsigned)((n + BM - 1) / BM));
    k_gemm_fp64<<<grid, kThreads, 0, st>>>(A, lda, B, ldb, C, ldc, n, k, m);
    return launch_status();
}

}  // namespace blaz
