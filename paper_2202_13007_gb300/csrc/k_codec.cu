// k_codec.cu -- compressor kernels (Sec. II of "Compressed Matrix
// Computations", arXiv 2202.13007); the decompressor is in k_decompress.cu.
//
// Compression is bit-exact binary64: every operation is an explicit
// round-to-nearest intrinsic in the order fixed in include/blaz.h, so the
// result does not depend on -fmad or on the compiler's scheduling.  The
// compressor runs in three launches: k_compress_fast<.., true> compresses
// the uniform blocks (one sign and one exponent field: Eq. eqnorm and the
// slope sum exact in integer arithmetic, compress_fast.cuh) and lists the
// others; k_compress_fast<.., false> compresses the listed blocks with the
// binary64 normalization, densely; both decide every code they can certify
// and list the codes (or whole blocks) they cannot, and k_compress_fix
// evaluates those exactly in binary64, densely, by teams of 8 lanes, so the
// rare exact work costs no divergence.
#include <mutex>

#include "compress_fast.cuh"
#include "compress_fix.cuh"
#include "gmap.cuh"

namespace blaz {

// Warp-aggregated append of `value` for the lanes where `want` holds.
template <typename T>
__device__ __forceinline__ void append(bool want, T value, T *__restrict__ list, unsigned *__restrict__ count)
{
    const unsigned act = __activemask();
    const unsigned need = __ballot_sync(act, want);
    if (!need) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(need) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned)__popc(need));
    base = __shfl_sync(act, base, leader);
    if (want) list[base + __popc(need & ((1u << lane) - 1u))] = value;
}

// CTA size of the fast compressor: 128 threads (one block each).  Both
// passes run 3 CTAs per SM: the uniform pass in 161 registers without spills
// (D leaves the registers row by row during the DCT), the binary64 pass in
// 168 with ~100 bytes of spills, which measured faster than 2 CTAs at 224
// registers.  Both are bound by instruction issue and latency rather than
// by the binary64 pipe.  The sign-coherent blocks of a CTA share one dense
// pass of exact DC chains, which larger CTAs fill better.
constexpr int kFastThreads = 128;

// Dynamic shared memory of the fast compressor: one slot per block of the
// CTA (the block, r = RN(1/s) and the meta word), the exact X00 of every
// slot, then a copy of the block's N (uniform pass) or D (binary64 pass) in
// an odd row of kSlot doubles (conflict-free row reads) for the first
// kCopySlots slots only.  The dense pass reloads the two rows each team lane
// needs for the other slots (cf_exact_dc_team_uniform, cf_exact_dc_team_d),
// so no block leaves a pass for lack of room.  A CTA needs 54 KB instead of
// 70, and the SM keeps 60 KB or more of L1 instead of ~28 KB, which also
// bounds the block loads in flight (a warp loads 16 KB per round) and holds
// the binary64 pass's spills; few CTAs of a smooth field have more than 96
// sign-coherent blocks.  Measured at 16384^2 on the uniform pass: 1.276 /
// 1.181 ms per compression of the two bump fields with 128 copied slots,
// 1.203 / 1.097 with 96 (with 32-byte loads), 1.253 / 1.104 with every slot
// reloaded; the binary64 pass's 96 copies took another 0.002-0.004 ms off.
constexpr int kSlot = 67;
constexpr int kCopySlots = 96;
struct FastSlot {
    double r;
    unsigned b, meta;
};
constexpr size_t kFastSmem =
    (sizeof(FastSlot) + sizeof(double)) * (size_t)kFastThreads + sizeof(double) * (size_t)kCopySlots * kSlot;

// X00 by a team for a block of the binary64 pass, from the input itself:
// lane u forms row u of D as compress_block does (team_d_row).
__device__ __forceinline__ double cf_exact_dc_team_d(const double *__restrict__ A, int64_t lda, int64_t rows,
                                                     int64_t cols, int64_t nbc, int64_t b, double r, int u,
                                                     unsigned tmask, int tbase)
{
    double dr[8];
    team_d_row(A, lda, rows, cols, nbc, b, u, dr);
    return cf_exact_dc_rows([&](int v) { return dr[v]; }, r, tmask, tbase);
}

// A full block with 32-byte loads: two per row of 64 B, so that every load
// instruction of a warp uses whole 32-byte sectors (with 16-byte loads two
// instructions share each sector).  Needs the base 32-byte aligned and lda
// a multiple of 4 (compress_ld_width).
__device__ __forceinline__ void load_block_wide(const double *__restrict__ A, int64_t lda, int64_t bi, int64_t bj,
                                                double (&d)[64])
{
    const double *p = A + (bi * 8) * lda + bj * 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double *q = p + i * lda + 4 * h;
            asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
                : "=d"(d[i * 8 + 4 * h]), "=d"(d[i * 8 + 4 * h + 1]), "=d"(d[i * 8 + 4 * h + 2]),
                  "=d"(d[i * 8 + 4 * h + 3])
                : "l"(q));
        }
    }
}

// One CTA's pass over up to kFastThreads blocks (thread t: block b when
// `valid`).  kUniform: the first pass, which compresses the uniform blocks
// on the integer pipe (cf_prepare_uniform) and lists every other block for
// the second pass (general_list); otherwise the second pass, on the binary64
// pipe (cf_prepare).  Both leave undecided codes and blocks to the fix-up
// lists.  Every thread of the CTA calls this (it holds barriers).  kLd: the
// width of the block loads, 0 scalar, 1 16 bytes, 2 32 bytes.
template <int kLd, bool kUniform>
__device__ __forceinline__ void compress_pass(const double *__restrict__ A, int64_t lda, int64_t rows, int64_t cols,
                                              int64_t nbc, int64_t b, bool valid, double *__restrict__ f,
                                              double *__restrict__ s, uint8_t *__restrict__ phi,
                                              int8_t *__restrict__ code, uint2 *__restrict__ code_list,
                                              unsigned *__restrict__ code_count, unsigned *__restrict__ block_list,
                                              unsigned *__restrict__ block_count, unsigned *__restrict__ general_list,
                                              unsigned *__restrict__ general_count, double *smem,
                                              unsigned &sCount)
{
    FastSlot *uS = reinterpret_cast<FastSlot *>(smem);
    double *sX = reinterpret_cast<double *>(uS + kFastThreads);
    double(*sD)[kSlot] = reinterpret_cast<double(*)[kSlot]>(sX + kFastThreads);  // N or D, first kCopySlots
    double d[64];
    double sv = 0.0;
    FastCtx ctx;
    ctx.state = 1u;
    ctx.coherent = false;
    int slot = -1;
    // A block that may need the exact DC chain takes a slot as soon as it is
    // normalized; r follows once s is known.
    auto stash = [&](const double (&dd)[64], unsigned meta) {
        slot = (int)atomicAdd(&sCount, 1u);
        uS[slot].b = (unsigned)b;
        uS[slot].meta = meta;
        if (slot < kCopySlots) {
#pragma unroll
            for (int p = 0; p < 64; ++p) sD[slot][p] = dd[p];
        }
    };
    if (valid) {
        const int64_t bi = b / nbc, bj = b - (b / nbc) * nbc;
        if (bi * 8 + 8 <= rows && bj * 8 + 8 <= cols) {
            if (kLd == 2) load_block_wide(A, lda, bi, bj, d);
            else load_block<kLd == 1>(A, lda, bi, bj, d);
        } else {
            load_block_clamped(A, lda, bi, bj, rows, cols, d);  // partial block of a padded matrix
        }
        const double f0 = d[0];
        if (kUniform) {
            valid = cf_prepare_uniform(d, sv, ctx, stash);
            append(!valid, (unsigned)b, general_list, general_count);
        } else {
            cf_prepare(d, sv, ctx, stash);
        }
        // r = RN(1/s) for the dense pass, formed here, where it overlaps the
        // other warps' work, rather than at the head of the team's chain
        // (1.205 / 1.101 -> 1.182 / 1.100 ms at 16384^2, 0.220 -> 0.203 ms
        // for a 4096^2 field of sign-coherent blocks)
        if (slot >= 0) uS[slot].r = ddiv(1.0, sv);
        if (valid) {
            f[b] = f0;
            s[b] = sv;
        }
    }
    __syncthreads();
    // the exact DC chains of the slots, one team of 8 lanes per slot (teams
    // never straddle a warp; a team is wholly active or idle)
    {
        const unsigned n = sCount;
        const int lane = threadIdx.x & 31, u = lane & 7, tbase = lane & ~7;
        const unsigned tmask = 0xFFu << tbase;
        for (unsigned w = threadIdx.x; w < 8u * n; w += blockDim.x) {
            const unsigned q = w >> 3;
            const double r = uS[q].r;
            double x;
            if (q < (unsigned)kCopySlots)
                x = kUniform ? cf_exact_dc_team_n(sD[q], r, uS[q].meta, u, tmask, tbase)
                             : cf_exact_dc_team(sD[q], r, u, tmask, tbase);
            else
                x = kUniform ? cf_exact_dc_team_uniform(A, lda, rows, cols, nbc, uS[q].b, r, uS[q].meta, u, tmask, tbase)
                             : cf_exact_dc_team_d(A, lda, rows, cols, nbc, uS[q].b, r, u, tmask, tbase);
            if (u == 0) sX[q] = x;
        }
    }
    __syncthreads();
    if (valid) {
        uint8_t ph = 255;
        uint32_t cw[7];
        const uint32_t pending = cf_finish(ctx, slot >= 0 ? sX[slot] : 0.0, ph, cw);
        if (pending != kPendingAll) {
            phi[b] = ph;
            uint32_t *w = reinterpret_cast<uint32_t *>(code + b * kKeep);  // 28 bytes, 4-byte aligned
#pragma unroll
            for (int q = 0; q < 7; ++q) w[q] = cw[q];
        }
        // Undecided codes and whole blocks go to separate lists, so that the
        // fix-up kernel runs without divergence between the two cases.
        append(pending != 0u && pending != kPendingAll, make_uint2((unsigned)b, pending), code_list, code_count);
        append(pending == kPendingAll, (unsigned)b, block_list, block_count);
    }
}

// The certified compressor.  kUniform: one CTA per kFastThreads consecutive
// blocks, the first pass of compress_pass.  Otherwise the second pass over
// the blocks the first one listed, the CTAs striding over the list.
template <int kLd, bool kUniform>
__global__ void __launch_bounds__(kFastThreads, 3)
    k_compress_fast(const double *__restrict__ A, int64_t lda, int64_t rows, int64_t cols, int64_t nbc, int64_t nb,
                    double *__restrict__ f, double *__restrict__ s, uint8_t *__restrict__ phi,
                    int8_t *__restrict__ code, uint2 *__restrict__ code_list, unsigned *__restrict__ code_count,
                    unsigned *__restrict__ block_list, unsigned *__restrict__ block_count,
                    unsigned *__restrict__ general_list, unsigned *__restrict__ general_count)
{
    // Sign-coherent blocks of the CTA take slots here; after a barrier teams
    // of the CTA's threads evaluate their exact DC chains densely and leave
    // X00 beside the slots (dynamic shared memory).
    extern __shared__ double fast_smem[];
    __shared__ unsigned sCount;
    if (kUniform) {
        if (threadIdx.x == 0) sCount = 0u;
        __syncthreads();
        const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        compress_pass<kLd, true>(A, lda, rows, cols, nbc, b, b < nb, f, s, phi, code, code_list, code_count,
                                  block_list, block_count, general_list, general_count, fast_smem, sCount);
    } else {
        const int64_t n = *general_count;  // the first pass completed before this launch
        for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
            if (threadIdx.x == 0) sCount = 0u;
            __syncthreads();
            const int64_t i = base + threadIdx.x;
            const int64_t b = i < n ? (int64_t)general_list[i] : 0;
            compress_pass<kLd, false>(A, lda, rows, cols, nbc, b, i < n, f, s, phi, code, code_list, code_count,
                                       block_list, block_count, general_list, general_count, fast_smem, sCount);
            __syncthreads();  // sCount and the shared slots are reused by the next chunk
        }
    }
}

// The exact fix-up of both lists in one launch: the whole-block list by
// teams of 8 lanes (fix_whole_block), then the undecided codes by one lane
// per block (fix_codes_lane).  The two lists hold different blocks, so the
// entries are independent.
template <bool kVec>
__global__ void __launch_bounds__(128)
    k_compress_fix(const double *__restrict__ A, int64_t lda, int64_t rows, int64_t cols, int64_t nbc,
                   const unsigned *__restrict__ block_list,
                   const uint2 *__restrict__ code_list, const unsigned *__restrict__ counts,
                   const double *__restrict__ s, uint8_t *__restrict__ phi, int8_t *__restrict__ code)
{
    __shared__ double cs[64];
    if (threadIdx.x < 64) cs[threadIdx.x] = c_cos[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, u = lane & 7, tbase = lane & ~7;
    const unsigned tmask = 0xFFu << tbase;
    const int64_t ncodes = counts[0], nblocks = counts[1];
    const int64_t threads = (int64_t)gridDim.x * blockDim.x, tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t q = tid / 8; q < nblocks; q += threads / 8)
        fix_whole_block<kVec>(A, lda, rows, cols, nbc, block_list[q], s, phi, code, u, tbase, tmask);
    for (int64_t q = tid; q < ncodes; q += threads) {
        const uint2 e = code_list[q];
        fix_codes_lane<kVec>(A, lda, rows, cols, nbc, e.x, e.y, s, phi, code, cs);
    }
}

static bool vec_ok(const void *p, int64_t ld) { return ((uintptr_t)p % 16 == 0) && (ld % 2 == 0); }

// One block per thread: short-lived CTAs keep the warps of an SM at different
// phases of the block (binary64 normalization, fp32 DCT, integer codes), so
// the FP64 pipe overlaps the others; a single resident wave of long-lived
// CTAs runs ~10% slower at 16384^2.
static int fast_grid(int64_t nb)
{
    const int64_t want = (nb + kFastThreads - 1) / kFastThreads;
    return (int)(want < 1 ? 1 : (want > 0x7FFFFFFF ? 0x7FFFFFFF : want));
}

// Scratch of one compression: the undecided-code list (8 B per entry), the
// whole-block list and the list of blocks for the second pass (4 B each),
// then the three counts.
size_t compress_scratch_bytes(int64_t nb)
{
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    return up((size_t)nb * 8) + 2 * up((size_t)nb * 4) + 256;
}

// The widest block load that every full block of A allows: 32 bytes when
// the base is 32-byte aligned and lda a multiple of 4 (every row of every
// block then starts on a 32-byte boundary), 16 bytes for 16 and 2, else 8.
static int compress_ld_width(const void *p, int64_t ld)
{
    if ((uintptr_t)p % 32 == 0 && ld % 4 == 0) return 2;
    return vec_ok(p, ld) ? 1 : 0;
}

template <int kLd>
static void compress_launches(const double *A, int64_t lda, int64_t rows, int64_t cols, int64_t nbc, int64_t nb,
                              const blaz_cmat *out, uint2 *code_list, unsigned *block_list, unsigned *general_list,
                              unsigned *counts, cudaStream_t st)
{
    // counts[0]: undecided codes, [1]: whole blocks, [2]: second-pass blocks
    k_compress_fast<kLd, true><<<fast_grid(nb), kFastThreads, kFastSmem, st>>>(
        A, lda, rows, cols, nbc, nb, out->f, out->s, out->phi, out->code, code_list, counts, block_list, counts + 1,
        general_list, counts + 2);
    // the second pass strides over its list (at most nb blocks) with up to
    // two resident waves of CTAs
    const int64_t want = (nb + kFastThreads - 1) / kFastThreads, cap = (int64_t)num_sms() * 6;
    k_compress_fast<kLd, false><<<(int)(want < cap ? want : cap), kFastThreads, kFastSmem, st>>>(
        A, lda, rows, cols, nbc, nb, out->f, out->s, out->phi, out->code, code_list, counts, block_list, counts + 1,
        general_list, counts + 2);
    k_compress_fix<(kLd > 0)><<<num_sms() * 4, 128, 0, st>>>(A, lda, rows, cols, nbc, block_list, code_list, counts,
                                                              out->s, out->phi, out->code);
}

// Both passes need more than the default 48 KB of dynamic shared memory per
// CTA.
template <int kLd>
static bool compress_smem_attribute()
{
    return cudaFuncSetAttribute(k_compress_fast<kLd, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kFastSmem) == cudaSuccess &&
           cudaFuncSetAttribute(k_compress_fast<kLd, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kFastSmem) == cudaSuccess;
}

int launch_compress(const double *A, int64_t lda, int64_t rows, int64_t cols, const blaz_cmat *out, void *scratch,
                    cudaStream_t st)
{
    const int64_t nbc = out->cols / 8, nb = (out->rows / 8) * nbc;
    if (nb == 0) return BLAZ_OK;
    if (nb > 0xFFFFFFFFll) return BLAZ_ERR_SHAPE;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    uint2 *code_list = (uint2 *)scratch;
    unsigned *block_list = (unsigned *)((char *)scratch + up((size_t)nb * 8));
    unsigned *general_list = (unsigned *)((char *)scratch + up((size_t)nb * 8) + up((size_t)nb * 4));
    unsigned *counts = (unsigned *)((char *)scratch + up((size_t)nb * 8) + 2 * up((size_t)nb * 4));
    cudaError_t e = cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned), st);
    if (e != cudaSuccess) return set_cuda_error(e);
    static const bool smem_ok =
        compress_smem_attribute<0>() && compress_smem_attribute<1>() && compress_smem_attribute<2>();
    if (!smem_ok) return set_cuda_error(cudaGetLastError());
    switch (compress_ld_width(A, lda)) {
    case 2: compress_launches<2>(A, lda, rows, cols, nbc, nb, out, code_list, block_list, general_list, counts, st); break;
    case 1: compress_launches<1>(A, lda, rows, cols, nbc, nb, out, code_list, block_list, general_list, counts, st); break;
    default: compress_launches<0>(A, lda, rows, cols, nbc, nb, out, code_list, block_list, general_list, counts, st);
    }
    return launch_status();
}

}  // namespace blaz
