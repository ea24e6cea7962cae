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

namespace blaz {

__device__ int g_device_status;  // 0 or a BLAZ_ERR_* code set by a kernel

namespace tc {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int kThreads = 192;  // warp 0: TMA producer, warp 1: MMA issuer, warps 2-5: epilogue
constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = BN;  // fp32 accumulator: 128 lanes x 256 columns
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false (and the status word set) when the limit runs out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            atomicExch(&g_device_status, BLAZ_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row x 128-byte atoms 1024 bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // SWIZZLE_128B
    return d;
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = BN, M = BM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

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
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {  // the whole warp allocates the accumulator columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
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
                mma_bf16(tmem_base, smem_desc(sa + kk * 32), smem_desc(sb + kk * 32), (kb | kk) != 0);
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS));
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
