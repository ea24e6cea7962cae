// k_mm_bf16.cu -- split-precision path of the compressed matrix product
// ("Matrix multiplication", Sec. III of "Compressed Matrix Computations",
// arXiv 2202.13007) on the 5th-generation tensor cores of sm_103a.
//
// A_hat (decompressed once) and B are each split into three bf16 slices,
// X ~ X1 + X2 + X3 (each slice the bf16 rounding of the remainder).  The six
// slice products with i + j <= 4,
//     A1B1 + A1B2 + A2B1 + A1B3 + A2B2 + A3B1,
// are one bf16 GEMM with an inner dimension of 6k: A' = [A1 A1 A2 A1 A2 A3]
// (n x 6k) times B' = [B1; B2; B1; B3; B2; B1] (6k x m, stored transposed,
// K-major).  The GEMM is a tcgen05.mma kernel: TMA loads 128x64 and 256x64
// bf16 tiles (128-byte swizzle) through a 4-stage mbarrier pipeline, one
// thread issues the MMAs into a 128x256 fp32 accumulator in tensor memory,
// four warps read it back with tcgen05.ld and store binary64.
//
// Every mbarrier wait is bounded; on expiry the kernel records
// BLAZ_ERR_TIMEOUT in the device status word, skips its remaining work,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "blaz_internal.cuh"
#include "tcgen05.cuh"

namespace blaz {

__device__ int g_device_status;  // 0 or a BLAZ_ERR_* code set by a kernel

namespace tc {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int kThreads = 192;  // warp 0: TMA producer, warp 1: MMA issuer, warps 2-5: epilogue
constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = BN;  // fp32 accumulator: 128 lanes x 256 columns
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

using namespace umma;

// Bounded wait recording a timeout in this library's device status word.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    return umma::mbar_wait(bar, parity, abort_flag, &g_device_status);
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// bf16 A and B, fp32 accumulator, N = BN, M = BM.
constexpr uint32_t kIdesc = idesc_f16(BM, BN, true, true);

// C (n x m, binary64, ldc) = A' (n x K, bf16, K-major) * B'^T (m x K, bf16, K-major)^T
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_bf16_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, double *C,
                   int64_t ldc, int n, int m, int K)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + (size_t)STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accum = empty + STAGES;
    uint32_t *tmem_slot = (uint32_t *)(accum + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM;  // rows of C (and of A')
    const int n0 = blockIdx.x * BN;  // columns of C (rows of B'^T)
    const int nkb = (K + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 1) {  // the whole warp allocates the accumulator columns
        tmem_alloc(tmem_slot, TMEM_COLS);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % STAGES;
            const uint32_t parity = ((kb / STAGES) & 1) ^ 1;
            if (!mbar_wait(&empty[s], parity, abort_flag)) break;
            uint8_t *sa = smem + (size_t)s * STAGE_BYTES;
            uint8_t *sb = sa + A_BYTES;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(sa, &map_a, &full[s], kb * BK, m0);
            tma_load_2d(sb, &map_b, &full[s], kb * BK, n0);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % STAGES;
            if (!mbar_wait(&full[s], (kb / STAGES) & 1, abort_flag)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + (size_t)s * STAGE_BYTES);
            const uint32_t sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_f16(tmem_base, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32), kIdesc, (kb | kk) != 0);
            mma_commit(&empty[s]);  // frees the stage when these MMAs complete
        }
        if (ok) mma_commit(accum);
    } else if (warp >= 2) {
        // Epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (rows of the tile).
        const int quarter = warp & 3;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(accum, 0, abort_flag));
        tc_fence_after();
        if (ok) {
            const int row = m0 + quarter * 32 + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, r);
                if (row < n) {
                    double *dst = C + (int64_t)row * ldc + n0 + c0;
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (n0 + c0 + q < m) dst[q] = (double)__uint_as_float(r[q]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// Slices of a binary64 value: x ~ x1 + x2 + x3, each the bf16 rounding of
// the remainder (computed in fp32, where the remainders are exact).
__device__ __forceinline__ void split3(double x, __nv_bfloat16 &x1, __nv_bfloat16 &x2, __nv_bfloat16 &x3)
{
    const float xf = (float)x;
    x1 = __float2bfloat16_rn(xf);
    const float r1 = xf - __bfloat162float(x1);
    x2 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(x2);
    x3 = __float2bfloat16_rn(r2);
}

// A' = [A1 A1 A2 A1 A2 A3]: n x 6k, row-major, from A (n x k, lda).
__global__ void k_split_a(const double *__restrict__ A, int64_t lda, int64_t n, int64_t k,
                          __nv_bfloat16 *__restrict__ Ap)
{
    const int64_t total = n * k;
    const int64_t K6 = 6 * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k, c = e - (e / k) * k;
        __nv_bfloat16 x1, x2, x3;
        split3(A[r * lda + c], x1, x2, x3);
        __nv_bfloat16 *row = Ap + r * K6 + c;
        row[0] = x1;
        row[k] = x1;
        row[2 * k] = x2;
        row[3 * k] = x1;
        row[4 * k] = x2;
        row[5 * k] = x3;
    }
}

// B'^T: m x 6k, row j = [B1[:,j] B2[:,j] B1[:,j] B3[:,j] B2[:,j] B1[:,j]],
// from B (k x m, ldb); 32 x 32 tiles transposed through shared memory.
__global__ void k_split_bt(const double *__restrict__ B, int64_t ldb, int64_t k, int64_t m, __nv_bfloat16 *__restrict__ Bt)
{
    __shared__ __nv_bfloat16 t1[32][33], t2[32][33], t3[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;  // column of B (row of B'^T)
    const int64_t r0 = (int64_t)blockIdx.y * 32;  // row of B (k index)
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int i = ty; i < 32; i += 8) {
        const int64_t r = r0 + i, c = c0 + tx;
        __nv_bfloat16 x1 = __float2bfloat16_rn(0.f), x2 = x1, x3 = x1;
        if (r < k && c < m) split3(B[r * ldb + c], x1, x2, x3);
        t1[i][tx] = x1;
        t2[i][tx] = x2;
        t3[i][tx] = x3;
    }
    __syncthreads();
    const int64_t K6 = 6 * k;
    for (int j = ty; j < 32; j += 8) {
        const int64_t col = c0 + j, kk = r0 + tx;
        if (col < m && kk < k) {
            __nv_bfloat16 *row = Bt + col * K6 + kk;
            row[0] = t1[tx][j];
            row[k] = t2[tx][j];
            row[2 * k] = t1[tx][j];
            row[3 * k] = t3[tx][j];
            row[4 * k] = t2[tx][j];
            row[5 * k] = t1[tx][j];
        }
    }
}

}  // namespace tc

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2-D bf16 tensor map over a rows x cols K-major matrix (row stride cols*2 bytes).
static int make_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, uint32_t box_rows)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return BLAZ_ERR_CUDA;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)tc::BK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? BLAZ_OK : BLAZ_ERR_CUDA;
}

// Reads and clears the device status word after synchronizing `st`.
// Self-test of the timeout path: one thread waits for a flag that nothing
// sets, for at most `max_cycles`, records BLAZ_ERR_TIMEOUT in the device
// status word and returns; the context stays usable.
__device__ unsigned g_probe_flag;  // never written

__global__ void k_probe_wait(long long max_cycles)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && !bounded_wait_geq(&g_probe_flag, 1u, max_cycles))
        atomicExch(&g_device_status, BLAZ_ERR_TIMEOUT);
}

int launch_probe_wait(int64_t max_cycles, cudaStream_t st)
{
    if (max_cycles < 0 || max_cycles > 4000000000LL) return BLAZ_ERR_ARG;
    k_probe_wait<<<1, 32, 0, st>>>((long long)max_cycles);
    return launch_status();
}

int device_status(cudaStream_t st)
{
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error(e);
    int v = 0;
    e = cudaMemcpyFromSymbol(&v, g_device_status, sizeof(int));
    if (e != cudaSuccess) return set_cuda_error(e);
    if (v != 0) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int));
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return v;
}

size_t split_bf16_scratch_bytes(int64_t n, int64_t k, int64_t m)
{
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return up((size_t)n * 6 * k * 2) + up((size_t)m * 6 * k * 2);
}

// C = A_hat * B with A_hat already decompressed (Ah, n x k, lda).  `scratch`
// holds split_bf16_scratch_bytes(n, k, m) bytes.
int launch_matmul_split_bf16(const double *Ah, int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc,
                             int64_t n, int64_t k, int64_t m, void *scratch, cudaStream_t st)
{
    if (n == 0 || m == 0) return BLAZ_OK;
    if (n > 0x7fffffff || m > 0x7fffffff || 6 * k > 0x7fffffff) return BLAZ_ERR_SHAPE;
    if (k == 0) {  // empty inner dimension: C = 0
        cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc * 8, 0, (size_t)m * 8, (size_t)n, st);
        return e == cudaSuccess ? BLAZ_OK : set_cuda_error(e);
    }
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    __nv_bfloat16 *Ap = (__nv_bfloat16 *)scratch;
    __nv_bfloat16 *Bt = (__nv_bfloat16 *)((char *)scratch + up((size_t)n * 6 * k * 2));
    const int64_t K6 = 6 * k;
    {
        const int64_t total = n * k;
        int64_t g = (total + 255) / 256;
        if (g > (int64_t)num_sms() * 32) g = (int64_t)num_sms() * 32;
        tc::k_split_a<<<(int)g, 256, 0, st>>>(Ah, lda, n, k, Ap);
        int rc = launch_status();
        if (rc) return rc;
        dim3 gb((unsigned)((m + 31) / 32), (unsigned)((k + 31) / 32));
        if (gb.y > 65535) return BLAZ_ERR_SHAPE;
        tc::k_split_bt<<<gb, dim3(32, 8), 0, st>>>(B, ldb, k, m, Bt);
        if ((rc = launch_status())) return rc;
    }
    CUtensorMap ma, mb;
    int rc;
    if ((rc = make_map(&ma, Ap, n, K6, tc::BM))) return rc;
    if ((rc = make_map(&mb, Bt, m, K6, tc::BN))) return rc;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tc::k_gemm_bf16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tc::SMEM_BYTES);
        if (e != cudaSuccess) return set_cuda_error(e);
        attr_set = true;
    }
    dim3 grid((unsigned)((m + tc::BN - 1) / tc::BN), (unsigned)((n + tc::BM - 1) / tc::BM));
    if (grid.y > 65535) return BLAZ_ERR_SHAPE;
    tc::k_gemm_bf16_tc<<<grid, tc::kThreads, tc::SMEM_BYTES, st>>>(ma, mb, C, ldc, (int)n, (int)m, (int)K6);
    return launch_status();
}

}  // namespace blaz
