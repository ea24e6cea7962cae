// k_matmul.cu -- dense products used by the compressed matrix product
// ("Matrix multiplication", Sec. III of "Compressed Matrix Computations",
// arXiv 2202.13007): the compressed operand is decompressed once into a
// stream-ordered scratch matrix, then multiplied here.
//
// FP64 path: mma.sync.m8n8k4.f64 (DMMA), the binary64 tensor instruction of
// sm_103a (tcgen05 has no f64 kind).
#include "gemm_fp64.cuh"

namespace blaz {

// C (n x m) = A (n x k) * B (k x m); row-major; n, k multiples of 8; any m >= 1.
__global__ void __launch_bounds__(kGemmThreads)
    k_gemm_fp64(const double *__restrict__ A, int64_t lda, const double *__restrict__ B, int64_t ldb,
                double *__restrict__ C, int64_t ldc, int64_t n, int64_t k, int64_t m)
{
    __shared__ GemmSmem sm;
    gemm_tile_fp64<false>(sm, A, lda, B, ldb, C, ldc, n, k, m, (int64_t)blockIdx.y * kGemmBM,
                          (int64_t)blockIdx.x * kGemmBN);
}

int launch_gemm_fp64(const double *A, int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc, int64_t n,
                     int64_t k, int64_t m, cudaStream_t st)
{
    if (n == 0 || m == 0) return BLAZ_OK;
    if ((n + kGemmBM - 1) / kGemmBM > 65535 || (m + kGemmBN - 1) / kGemmBN > 0x7fffffff) return BLAZ_ERR_SHAPE;
    dim3 grid((unsigned)((m + kGemmBN - 1) / kGemmBN), (unsigned)((n + kGemmBM - 1) / kGemmBM));
    k_gemm_fp64<<<grid, kGemmThreads, 0, st>>>(A, lda, B, ldb, C, ldc, n, k, m);
    return launch_status();
}

}  // namespace blaz
