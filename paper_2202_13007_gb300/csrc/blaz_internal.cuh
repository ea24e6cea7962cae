// blaz_internal.cuh -- device constants and helpers shared by the blaz CUDA
// kernels (GB300, sm_103a).  Block format and constants follow Sec. II/III of
// "Compressed Matrix Computations" (arXiv 2202.13007).
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/blaz.h"

namespace blaz {

constexpr int kKeep = BLAZ_NKEEP;  // 28 kept coefficients per block (Sec. II, Ex. 5)

// RN(cos((2x+1) k pi / 16)), k = row, x = column (Sec. III, Eq. eqdct).
// Correctly rounded binary64 values of the mathematical constants.
#define BLAZ_C1 0x1.f6297cff75cb0p-1   // cos(1 pi/16)
#define BLAZ_C2 0x1.d906bcf328d46p-1   // cos(2 pi/16)
#define BLAZ_C3 0x1.a9b66290ea1a3p-1   // cos(3 pi/16)
#define BLAZ_C4 0x1.6a09e667f3bcdp-1   // cos(4 pi/16)
#define BLAZ_C5 0x1.1c73b39ae68c8p-1   // cos(5 pi/16)
#define BLAZ_C6 0x1.87de2a6aea963p-2   // cos(6 pi/16)
#define BLAZ_C7 0x1.8f8b83c69a60bp-3   // cos(7 pi/16)
// RN(alpha_i alpha_j): alpha_0^2 = 1/8, alpha_0 alpha_k = sqrt(2)/8, alpha_k^2 = 1/4.
#define BLAZ_A00 0x1.0000000000000p-3
#define BLAZ_A0K 0x1.6a09e667f3bcdp-3
#define BLAZ_AKK 0x1.0000000000000p-2

// COS[k][x] as a compile-time table (used with constant indices only, so it
// folds into immediates).
__host__ __device__ constexpr double cos_tab(int k, int x)
{
#define C(a, b, c, d, e, f, g, h) \
    (x == 0 ? (a) : x == 1 ? (b) : x == 2 ? (c) : x == 3 ? (d) : x == 4 ? (e) : x == 5 ? (f) : x == 6 ? (g) : (h))
    return k == 0   ? 1.0
           : k == 1 ? C(BLAZ_C1, BLAZ_C3, BLAZ_C5, BLAZ_C7, -BLAZ_C7, -BLAZ_C5, -BLAZ_C3, -BLAZ_C1)
           : k == 2 ? C(BLAZ_C2, BLAZ_C6, -BLAZ_C6, -BLAZ_C2, -BLAZ_C2, -BLAZ_C6, BLAZ_C6, BLAZ_C2)
           : k == 3 ? C(BLAZ_C3, -BLAZ_C7, -BLAZ_C1, -BLAZ_C5, BLAZ_C5, BLAZ_C1, BLAZ_C7, -BLAZ_C3)
           : k == 4 ? C(BLAZ_C4, -BLAZ_C4, -BLAZ_C4, BLAZ_C4, BLAZ_C4, -BLAZ_C4, -BLAZ_C4, BLAZ_C4)
           : k == 5 ? C(BLAZ_C5, -BLAZ_C1, BLAZ_C7, BLAZ_C3, -BLAZ_C3, -BLAZ_C7, BLAZ_C1, -BLAZ_C5)
           : k == 6 ? C(BLAZ_C6, -BLAZ_C2, BLAZ_C2, -BLAZ_C6, -BLAZ_C6, BLAZ_C2, -BLAZ_C2, BLAZ_C6)
                    : C(BLAZ_C7, -BLAZ_C5, BLAZ_C3, -BLAZ_C1, BLAZ_C1, -BLAZ_C3, BLAZ_C5, -BLAZ_C7);
#undef C
}

__host__ __device__ constexpr double aa_tab(int i, int j)
{
    return (i == 0 && j == 0) ? BLAZ_A00 : (i == 0 || j == 0) ? BLAZ_A0K : BLAZ_AKK;
}

// Kept position t -> (row, col): row 0, row 1, then (i,0),(i,1) for i = 2..7.
__host__ __device__ constexpr int kept_row(int t) { return t < 16 ? t / 8 : 2 + (t - 16) / 2; }
__host__ __device__ constexpr int kept_col(int t) { return t < 16 ? t % 8 : (t - 16) % 2; }
// Inverse map: kept index of (i,j), or -1 when the coefficient is dropped.
__host__ __device__ constexpr int kept_index(int i, int j)
{
    return i < 2 ? i * 8 + j : (j < 2 ? 16 + (i - 2) * 2 + j : -1);
}

// Binary64 operations that the compiler may not fuse or reorder.
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// trunc toward zero, saturated to [-127, 127], NaN -> 0.
// S = sum |D| of Eqs. eqslope / eqslope2 as the fixed pairwise tree over the
// row-major index: q[k] = |D_k| + |D_k+32| (k < 32), then q[k] += q[k+h] for
// h = 16, 8, 4, 2, 1; S = q[0].  Depth 6.
__device__ __forceinline__ double tree_sum_abs(const double (&d)[64])
{
    double q[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) q[k] = dadd(fabs(d[k]), fabs(d[k + 32]));
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1)
#pragma unroll
        for (int k = 0; k < h; ++k) q[k] = dadd(q[k], q[k + h]);
    return q[0];
}

__device__ __forceinline__ int8_t quantize(double v)
{
    if (v != v) return 0;
    if (v >= 127.0) return 127;
    if (v <= -127.0) return -127;
    return (int8_t)__double2int_rz(v);
}

// The same function on the integer pipe (the binary64 pipe is the scarce
// one): trunc toward zero saturated to [-127, 127], NaN -> 0, from the bits.
__device__ __forceinline__ int8_t quantize_bits(double v)
{
    const long long b = __double_as_longlong(v);
    const bool neg = b < 0;
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0x7FF) return (b & 0x000FFFFFFFFFFFFFll) ? 0 : (neg ? -127 : 127);
    if (e < 1023) return 0;
    if (e >= 1023 + 7) return neg ? -127 : 127;
    const unsigned long long m = ((unsigned long long)b & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    int mag = (int)(m >> (52 - (e - 1023)));
    mag = mag > 127 ? 127 : mag;
    return (int8_t)(neg ? -mag : mag);
}

// Truncation toward zero to int8, saturated to [-128, 127] (the low byte of
// the result register).
__device__ __forceinline__ uint32_t cvt_s8_rz(float x)
{
    uint32_t r;
    asm("cvt.rzi.s8.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Bit 7 of byte k set when byte k of the truncations of the two ends differs,
// or when that of the lower end is -128 (0x80: saturated, below quantize's
// range): the undecided codes of a word.  Per byte x, (x & 0x7F) + 0x7F sets
// bit 7 exactly when the low 7 bits are not all zero, with no carry into the
// next byte.
__device__ __forceinline__ uint32_t undecided_bytes(uint32_t lw, uint32_t hw)
{
    const uint32_t d = lw ^ hw;
    const uint32_t ne = ((d & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | d;
    const uint32_t m128 = ~((lw & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) & lw;
    return (ne | m128) & 0x80808080u;
}

// ---- host-side launch plumbing (defined in blaz_api.cu) ------------------------
int set_cuda_error(cudaError_t e);   // records e, returns BLAZ_ERR_CUDA
int launch_status();                 // cudaGetLastError -> BLAZ_OK / BLAZ_ERR_CUDA
int num_sms();                       // SM count of the current device (cached)
int validate_cmat(const blaz_cmat *m);   // shape, NULL and alignment checks of a descriptor

// An NVTX range over a host call (visible in Nsight timelines; a few ns when
// no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
#define BLAZ_NVTX() ::blaz::NvtxRange blaz_nvtx_range_(__func__)

// Waits until *flag >= target for at most max_cycles SM clock cycles; false
// when the limit ran out (the caller records BLAZ_ERR_TIMEOUT and returns).
// Every spin-wait of the library goes through a bounded wait.
__device__ __forceinline__ bool bounded_wait_geq(const volatile unsigned *flag, unsigned target, long long max_cycles)
{
    const long long t0 = clock64();
    while (*flag < target)
        if (clock64() - t0 > max_cycles) return false;
    return true;
}

// Self-test of the device-side timeout path (k_mm_bf16.cu).
int launch_probe_wait(int64_t max_cycles, cudaStream_t st);

// Keeps the current device's default memory pool (this process's
// stream-ordered allocations) cached across synchronizations instead of
// returning it to the system, so that scratch and staging are re-used rather
// than re-mapped call after call.  Once per device.
void keep_pool_cached();

// Stream-ordered scratch that is released on the same stream.
struct Scratch {
    void *p = nullptr;
    cudaStream_t st;
    explicit Scratch(cudaStream_t s) : st(s) {}
    int alloc(size_t bytes)
    {
        keep_pool_cached();
        cudaError_t e = cudaMallocAsync(&p, bytes ? bytes : 16, st);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? BLAZ_ERR_OOM : set_cuda_error(e);
        }
        return BLAZ_OK;
    }
    ~Scratch()
    {
        if (p) cudaFreeAsync(p, st);
    }
};
int batch_device_status();           // reads and clears the batch kernel's status word
int ops_device_status();             // reads and clears the tiled addition's status word

// ---- launchers (one per kernel family) ------------------------------------------
size_t compress_scratch_bytes(int64_t nb);
// rows x cols: the logical shape (rows, cols >= 1 when out has blocks); blocks
// beyond it read the edge-replicated extension.
int launch_compress(const double *A, int64_t lda, int64_t rows, int64_t cols, const blaz_cmat *out, void *scratch,
                    cudaStream_t st);
// rows x cols: the logical shape (-1: the block grid's); entries of partial
// blocks beyond it are skipped, or written as 0 when zero_fill is set.
int launch_decompress(const blaz_cmat *a, double *A, int64_t lda, cudaStream_t st, int64_t rows = -1,
                      int64_t cols = -1, bool zero_fill = false);
// The split-precision product's A operand straight from the codes: the three
// bf16 slices of A_hat into Sl = [A1 A2 A3] (rows x 3kp), padding zeroed.
int launch_decompress_slices(const blaz_cmat *a, void *Sl, int64_t kp, cudaStream_t st);
int launch_add(const blaz_cmat *a, const blaz_cmat *b, const blaz_cmat *out, bool subtract, cudaStream_t st);
int launch_scale(const blaz_cmat *a, double c, const blaz_cmat *out, cudaStream_t st);
// rows x cols: the logical shape (-1: the block grid's); for a padded pair the
// partial blocks are summed over their logical entries by a second kernel.
int launch_dot(const blaz_cmat *a, const blaz_cmat *b, double *result, double *partials, unsigned *counter,
               int64_t max_ctas, cudaStream_t st, int64_t rows = -1, int64_t cols = -1);
// Largest grid of the flattened dot (k_dot_tc): one partial sum per CTA, so
// this is also the number of partial-sum slots every caller provides.
constexpr int kDotMaxCtas = 1024;
int dot_grid(int64_t nb);
int rowcol_grid(int64_t nkb);
int launch_dot_rowcol(const blaz_cmat *a, const blaz_cmat *b, int64_t i, int64_t j, double *result,
                      double *partials, unsigned *counter, cudaStream_t st);
size_t split_bf16_scratch_bytes(int64_t n, int64_t k, int64_t m);
int launch_gemm_split_bf16(const void *Ap, const void *Bt, double *C, int64_t ldc, int64_t n, int64_t m, int64_t kp,
                           cudaStream_t st);
int launch_matmul_split_bf16_cmat(const blaz_cmat *a, const double *B, int64_t ldb, double *C, int64_t ldc,
                                  int64_t m, void *scratch, cudaStream_t st);
int launch_matmul_split_bf16(const double *Ah, int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc,
                             int64_t n, int64_t k, int64_t m, void *scratch, cudaStream_t st);
int device_status(cudaStream_t st);
int launch_gemm_fp64(const double *A, int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc,
                     int64_t n, int64_t k, int64_t m, cudaStream_t st);

}  // namespace blaz
