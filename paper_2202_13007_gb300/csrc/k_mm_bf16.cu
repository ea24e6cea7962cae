// k_mm_bf16.cu -- split-precision path of the compressed matrix product
// ("Matrix multiplication", Sec. III of "Compressed Matrix Computations",
// arXiv 2202.13007) on the 5th-generation tensor cores of sm_103a.
//
// A_hat (decompressed once) and B are each split into three bf16 slices,
// X ~ X1 + X2 + X3 (each slice the bf16 rounding of the remainder).  The six
// slice products with i + j <= 4,
//     A1B1 + A1B2 + A2B1 + A1B3 + A2B2 + A3B1,
// are one bf16 GEMM with an inner dimension of six segments of kp columns
// (kp: k rounded up to the 64-column K tile, the padding zero): segment g
// multiplies slice kSliceA[g] of A' = [A1 A2 A3] (n x 3kp) by slice
// kSliceB[g] of B'^T = [B1 B2 B3] (m x 3kp, K-major).  Only the three slices
// are stored, once each; the TMA producer maps every K tile to its slice,
// and the repeated slices are read again from L2.  The GEMM is a
// tcgen05.mma kernel: TMA loads 128x64 and 256x64 bf16 tiles (128-byte
// swizzle) through a 4-stage mbarrier pipeline, one thread issues the MMAs
// into a 128x256 fp32 accumulator in tensor memory, four warps read it back
// with tcgen05.ld and store binary64.
//
// Every mbarrier wait is bounded; on expiry the kernel records
// BLAZ_ERR_TIMEOUT in the device status word, skips its remaining work,
// frees its tensor memory and returns.
#include <cuda.h>
#include <mutex>
#include <vector>
#include <cuda_bf16.h>

#include "blaz_internal.cuh"
#include "split_bf16.cuh"
#include "tcgen05.cuh"

namespace blaz {

__device__ int g_device_status;  // 0 or a BLAZ_ERR_* code set by a kernel

namespace tc {

constexpr int BM = 128, BK = 64;
constexpr int kThreads = 192;  // warp 0: TMA producer, warp 1: MMA issuer, warps 2-5: epilogue
constexpr uint32_t A_BYTES = BM * BK * 2;
constexpr size_t kSmemMax = 227 * 1024;

// A tile of BM x BN outputs: N = BN columns (a multiple of 32, at most 256),
// as many pipeline stages as fit in shared memory (at most 8), and the
// accumulator's tensor-memory columns rounded up to a power of two.
template <int BN>
struct Tile {
    static constexpr uint32_t B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int STAGES_FIT = (int)((kSmemMax - 1024 - 256) / STAGE_BYTES);
    static constexpr int STAGES = STAGES_FIT > 8 ? 8 : STAGES_FIT;
    static constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    static constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
    static constexpr uint32_t IDESC = umma::idesc_f16(BM, BN, true, true);  // bf16 A and B, fp32 accumulator
    static_assert(BN % 32 == 0 && BN <= 256 && STAGES >= 2, "tile shape");
};

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

// Slice of A' and of B'^T that K segment g multiplies (levels i + j <= 4).
__device__ __forceinline__ int slice_a(int g) { return g == 2 || g == 4 ? 1 : g == 5 ? 2 : 0; }
__device__ __forceinline__ int slice_b(int g) { return g == 1 || g == 4 ? 1 : g == 3 ? 2 : 0; }

// C (n x m, binary64, ldc) = sum over the six K segments g of
// A'[:, slice_a(g)] (n x kp) * B'^T[:, slice_b(g)]^T; kbs = kp / BK tiles per
// segment.
template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_bf16_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, double *C,
                   int64_t ldc, int n, int m, int kbs)
{
    using T = Tile<BN>;
    constexpr int STAGES = T::STAGES;
    constexpr uint32_t STAGE_BYTES = T::STAGE_BYTES, TMEM_COLS = T::TMEM_COLS;
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
    const int nkb = 6 * kbs;

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
            const int g = kb / kbs, kt = kb - g * kbs;
            tma_load_2d(sa, &map_a, &full[s], (slice_a(g) * kbs + kt) * BK, m0);
            tma_load_2d(sb, &map_b, &full[s], (slice_b(g) * kbs + kt) * BK, n0);
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
                mma_f16(tmem_base, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32), T::IDESC,
                        (kb | kk) != 0);
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

// A' = [A1 A2 A3]: n x 3kp, row-major, from A (n x k, lda); columns k..kp-1
// of each slice are zero.
__global__ void k_split_a(const double *__restrict__ A, int64_t lda, int64_t n, int64_t k, int64_t kp,
                          __nv_bfloat16 *__restrict__ Ap)
{
    const int64_t total = n * kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / kp, c = e - (e / kp) * kp;
        __nv_bfloat16 x1 = __float2bfloat16_rn(0.f), x2 = x1, x3 = x1;
        if (c < k) split3(A[r * lda + c], x1, x2, x3);
        __nv_bfloat16 *row = Ap + r * 3 * kp + c;
        row[0] = x1;
        row[kp] = x2;
        row[2 * kp] = x3;
    }
}

// B'^T = [B1 B2 B3]: m x 3kp, row j the three slices of column j of B (k x m,
// ldb), zero beyond k; 32 x 32 tiles transposed through shared memory.
__global__ void k_split_bt(const double *__restrict__ B, int64_t ldb, int64_t k, int64_t kp, int64_t m,
                           __nv_bfloat16 *__restrict__ Bt)
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
    for (int j = ty; j < 32; j += 8) {
        const int64_t col = c0 + j, kk = r0 + tx;
        if (col < m && kk < kp) {
            __nv_bfloat16 *row = Bt + col * 3 * kp + kk;
            row[0] = t1[tx][j];
            row[kp] = t2[tx][j];
            row[2 * kp] = t3[tx][j];
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

static int launch_split_bt(const double *B, int64_t ldb, int64_t k, int64_t kp, int64_t m, __nv_bfloat16 *Bt,
                           cudaStream_t st);

// A second stream per device on which the B operand's slices are formed
// while the caller's stream forms A's (the two are independent).
static cudaStream_t aux_stream()
{
    static std::mutex mu;
    static std::vector<cudaStream_t> streams;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)streams.size() <= dev) streams.resize(dev + 1, nullptr);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
        streams[dev] = nullptr;
    return streams[dev];
}

// Runs on_aux(aux) on the auxiliary stream and on_st() on st concurrently:
// aux starts after st's earlier work (the scratch allocation), st continues
// after both.  Fork and join by events, so stream capture sees one graph.
template <typename FA, typename FS>
static int fork_join(cudaStream_t st, FA on_aux, FS on_st)
{
    cudaStream_t ax = aux_stream();
    if (!ax) return BLAZ_ERR_CUDA;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ax, ev[0], 0);
    int rc = e == cudaSuccess ? on_aux(ax) : set_cuda_error(e);
    // join even after a failure, so that st never runs ahead of work on ax
    const int rs = rc == BLAZ_OK ? on_st() : BLAZ_OK;
    e = cudaEventRecord(ev[1], ax);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[1], 0);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (rc) return rc;
    if (rs) return rs;
    return e == cudaSuccess ? BLAZ_OK : set_cuda_error(e);
}

// k rounded up to the GEMM's K tile (each slice is padded to it).
static int64_t split_kp(int64_t k) { return (k + tc::BK - 1) / tc::BK * tc::BK; }

size_t split_bf16_scratch_bytes(int64_t n, int64_t k, int64_t m)
{
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const int64_t kp = split_kp(k);
    return up((size_t)n * 3 * kp * 2) + up((size_t)m * 3 * kp * 2);
}

// C = A_hat * B with A_hat already decompressed (Ah, n x k, lda).  `scratch`
// holds split_bf16_scratch_bytes(n, k, m) bytes.
int launch_matmul_split_bf16(const double *Ah, int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc,
                             int64_t n, int64_t k, int64_t m, void *scratch, cudaStream_t st)
{
    if (n == 0 || m == 0) return BLAZ_OK;
    if (n > 0x7fffffff || m > 0x7fffffff || 6 * split_kp(k) > 0x7fffffff) return BLAZ_ERR_SHAPE;
    if (k == 0) {  // empty inner dimension: C = 0
        cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc * 8, 0, (size_t)m * 8, (size_t)n, st);
        return e == cudaSuccess ? BLAZ_OK : set_cuda_error(e);
    }
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const int64_t kp = split_kp(k);
    __nv_bfloat16 *Ap = (__nv_bfloat16 *)scratch;
    __nv_bfloat16 *Bt = (__nv_bfloat16 *)((char *)scratch + up((size_t)n * 3 * kp * 2));
    int rc = fork_join(
        st, [&](cudaStream_t ax) { return launch_split_bt(B, ldb, k, kp, m, Bt, ax); },
        [&]() {
            const int64_t total = n * kp;
            int64_t g = (total + 255) / 256;
            if (g > (int64_t)num_sms() * 32) g = (int64_t)num_sms() * 32;
            tc::k_split_a<<<(int)g, 256, 0, st>>>(Ah, lda, n, k, kp, Ap);
            return launch_status();
        });
    if (rc) return rc;
    return launch_gemm_split_bf16(Ap, Bt, C, ldc, n, m, kp, st);
}

// B'^T = [B1 B2 B3] (m x 3kp) from a dense B (k x m, ldb).
static int launch_split_bt(const double *B, int64_t ldb, int64_t k, int64_t kp, int64_t m, __nv_bfloat16 *Bt,
                           cudaStream_t st)
{
    dim3 gb((unsigned)((m + 31) / 32), (unsigned)((kp + 31) / 32));
    if (gb.y > 65535 || gb.x > 0x7fffffffu) return BLAZ_ERR_SHAPE;
    tc::k_split_bt<<<gb, dim3(32, 8), 0, st>>>(B, ldb, k, kp, m, Bt);
    return launch_status();
}

// C = A_hat * B with A_hat compressed (full blocks, n x k): A's slices come
// straight from the codes (no binary64 copy of A_hat), then B's, then the
// GEMM.  `scratch` holds split_bf16_scratch_bytes(n, k, m) bytes.
int launch_matmul_split_bf16_cmat(const blaz_cmat *a, const double *B, int64_t ldb, double *C, int64_t ldc,
                                  int64_t m, void *scratch, cudaStream_t st)
{
    const int64_t n = a->rows, k = a->cols;
    if (n == 0 || m == 0) return BLAZ_OK;
    if (n > 0x7fffffff || m > 0x7fffffff || 6 * split_kp(k) > 0x7fffffff) return BLAZ_ERR_SHAPE;
    if (k == 0) {  // empty inner dimension: C = 0
        cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc * 8, 0, (size_t)m * 8, (size_t)n, st);
        return e == cudaSuccess ? BLAZ_OK : set_cuda_error(e);
    }
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const int64_t kp = split_kp(k);
    __nv_bfloat16 *Ap = (__nv_bfloat16 *)scratch;
    __nv_bfloat16 *Bt = (__nv_bfloat16 *)((char *)scratch + up((size_t)n * 3 * kp * 2));
    int rc = fork_join(
        st, [&](cudaStream_t ax) { return launch_split_bt(B, ldb, k, kp, m, Bt, ax); },
        [&]() { return launch_decompress_slices(a, Ap, kp, st); });
    if (rc) return rc;
    return launch_gemm_split_bf16(Ap, Bt, C, ldc, n, m, kp, st);
}

template <int BN>
static int launch_gemm_tile(const CUtensorMap &ma, const CUtensorMap &mb, double *C, int64_t ldc, int64_t n,
                            int64_t m, int64_t kp, cudaStream_t st)
{
    using T = tc::Tile<BN>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tc::k_gemm_bf16_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)T::SMEM_BYTES);
        if (e != cudaSuccess) return set_cuda_error(e);
        attr_set = true;
    }
    dim3 grid((unsigned)((m + BN - 1) / BN), (unsigned)((n + tc::BM - 1) / tc::BM));
    if (grid.y > 65535) return BLAZ_ERR_SHAPE;
    tc::k_gemm_bf16_tc<BN><<<grid, tc::kThreads, T::SMEM_BYTES, st>>>(ma, mb, C, ldc, (int)n, (int)m,
                                                                       (int)(kp / tc::BK));
    return launch_status();
}

// The GEMM of the split product on slices already in place: Ap = [A1 A2 A3]
// (n x 3kp) and Bt = [B1 B2 B3] (m x 3kp), kp a multiple of the K tile.
int launch_gemm_split_bf16(const void *Ap, const void *Bt, double *C, int64_t ldc, int64_t n, int64_t m,
                           int64_t kp, cudaStream_t st)
{
    CUtensorMap ma, mb;
    int rc;
    if ((rc = make_map(&ma, Ap, n, 3 * kp, tc::BM))) return rc;
    // The tile width with the fewest column-waves of work: ceil(tiles / SMs)
    // x BN, the larger width on a tie (fewer operand bytes per product).
    const int64_t rt = (n + tc::BM - 1) / tc::BM, sms = num_sms();
    int bn = 256;
    int64_t best = -1;
    for (int cand : {256, 224, 192, 128}) {
        const int64_t waves = (rt * ((m + cand - 1) / cand) + sms - 1) / sms, cost = waves * cand;
        if (best < 0 || cost < best) {
            best = cost;
            bn = cand;
        }
    }
    if ((rc = make_map(&mb, Bt, m, 3 * kp, (uint32_t)bn))) return rc;
    switch (bn) {
    case 256: return launch_gemm_tile<256>(ma, mb, C, ldc, n, m, kp, st);
    case 224: return launch_gemm_tile<224>(ma, mb, C, ldc, n, m, kp, st);
    case 192: return launch_gemm_tile<192>(ma, mb, C, ldc, n, m, kp, st);
    default: return launch_gemm_tile<128>(ma, mb, C, ldc, n, m, kp, st);
    }
}

}  // namespace blaz
