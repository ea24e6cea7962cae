// k_decompress.cu -- the decompressor of "Compressed Matrix Computations"
// (arXiv 2202.13007, Sec. III, Eqs. eqbbb0 / eqbbb: inverse DCT of the kept
// coefficients scaled back by phi and s, then the inverse of the
// normalization of Eq. eqnorm), as a product with the fixed map G on the
// tensor cores.
#include <algorithm>
#include <cmath>
#include <mutex>

#include <cuda_fp16.h>

#include "blaz_internal.cuh"
#include "const_upload.cuh"
#include "gmap.cuh"
#include "split_bf16.cuh"

namespace blaz {

// ---------------------------------------------------------------------------------
// Decompression as a product with the fixed map G (gmap.cuh): Y = C G^T for 16
// blocks per warp on the tensor cores (mma.sync m16n8k16, fp16 inputs, fp32
// accumulation).  G is split into four fixed-point slices of 11 bits whose
// digits (|d| <= 2^10) and the codes (|c| <= 128) are exact in fp16; every
// product sum is an integer below 2^22 (28 * 2^7 * 2^10), exact in fp32 and
// within the range of the fp32 -> integer step below.  The assembly
//     Y = Y_0 2^33 + Y_1 2^22 + Y_2 2^11 + Y_3
// is exact in int64, and each output is one binary64 fma:
//     out = f + (s / phi) 2^E Y.
// G is represented to 2^-44 of its largest entry (1.75), so outputs differ
// from the binary64 evaluation of the definition by far less than 1e-12 of
// the block's scale |f| + 14 |s| sum|c| / phi.
constexpr int kDecSlices = 4;
constexpr int kDecDigitBits = 11;
struct DecConsts {
    uint2 bfrag[kDecSlices][2][8][32];  // B fragments [slice][k-step][n-tile][lane]
    double inv_phi_scaled[256];         // RN(1/phi) 2^E (2^E: weight of the last slice; exact scaling)
};
__device__ DecConsts g_dec;  // dec_consts(), copied once per device

static const DecConsts &dec_consts()
{
    static DecConsts dc;
    static std::once_flag once;
    std::call_once(once, [] {
        const long double(*G)[kKeep] = decompress_map();
        long double mx = 0.0L;
        for (int p = 0; p < 64; ++p)
            for (int t = 0; t < kKeep; ++t) mx = std::max(mx, fabsl(G[p][t]));
        const int E = (int)ceill(log2l(mx)) - (kDecDigitBits - 1);
        static float digit[kDecSlices][64][32];  // [slice][n = p][k = t], k >= 28 zero
        for (int p = 0; p < 64; ++p)
            for (int t = 0; t < 32; ++t) {
                long double r = t < kKeep ? G[p][t] : 0.0L;
                for (int s = 0; s < kDecSlices; ++s) {
                    const long double sc = ldexpl(1.0L, E - kDecDigitBits * s);
                    const long double d = rintl(r / sc);
                    digit[s][p][t] = (float)d;
                    r -= d * sc;
                }
            }
        auto h2 = [](float lo, float hi) {
            const __half a = __float2half_rn(lo), b = __float2half_rn(hi);
            return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
        };
        for (int s = 0; s < kDecSlices; ++s)
            for (int ks = 0; ks < 2; ++ks)
                for (int nt = 0; nt < 8; ++nt)
                    for (int lane = 0; lane < 32; ++lane) {
                        const int g = lane >> 2, t = lane & 3, n = nt * 8 + g, k = ks * 16 + 2 * t;
                        dc.bfrag[s][ks][nt][lane].x = h2(digit[s][n][k], digit[s][n][k + 1]);
                        dc.bfrag[s][ks][nt][lane].y = h2(digit[s][n][k + 8], digit[s][n][k + 9]);
                    }
        const double scale = (double)ldexpl(1.0L, E - kDecDigitBits * (kDecSlices - 1));
        dc.inv_phi_scaled[0] = 0.0;
        for (int p = 1; p < 256; ++p) dc.inv_phi_scaled[p] = (1.0 / (double)p) * scale;
    });
    return dc;
}

__device__ __forceinline__ void mma_f16(float (&c)[4], const uint32_t (&a)[4], uint2 b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// Two consecutive int8 codes (k, k+1) of a block as an fp16 pair; zero beyond
// 28.  Off the conversion unit: byte x ^ 0x80 = x + 128 under the exponent of
// 1024 is the fp16 number 1152 + x, and one exact subtraction leaves x.
__device__ __forceinline__ uint32_t code_pair(const int8_t *__restrict__ c, int k, bool valid)
{
    if (!valid || k >= kKeep) return 0u;
    const uint32_t v = __ldg(reinterpret_cast<const uint16_t *>(c + k));
    const uint32_t q = __byte_perm(v ^ 0x8080u, 0x64646464u, 0x4140);
    const __half2 h = __hsub2(*reinterpret_cast<const __half2 *>(&q), __half2half2(__ushort_as_half((unsigned short)0x6480)));
    return *reinterpret_cast<const uint32_t *>(&h);
}

static_assert(slice_assembly_bound(kDecSlices, kDecDigitBits, kKeep) < (1ull << 62),
              "the slice assembly must fit dec_to_double's input range");
static_assert((long long)kKeep * 128 * (1 << (kDecDigitBits - 1)) < (1ll << 22),
              "slice sums below 2^22 (exact in fp32 and in the fp32 -> int step)");

// kSlices: instead of the binary64 matrix, the three bf16 slices of every
// decoded value (split3) go to Sl = [A1 A2 A3] (rows x 3kp, row-major: the
// split-precision product's A operand); full blocks only.
template <bool kVec, bool kSlices = false>
__global__ void __launch_bounds__(128)
    k_decompress(const double *__restrict__ f, const double *__restrict__ s,
                 const uint8_t *__restrict__ phi, const int8_t *__restrict__ code, int64_t nbc, int64_t nb,
                 double *__restrict__ A, int64_t lda, int64_t rows, int64_t cols, bool zero_fill,
                 __nv_bfloat16 *__restrict__ Sl = nullptr, int64_t kp = 0)
{
    __shared__ uint2 sb[kDecSlices][2][8][32];
    __shared__ double inv_phi_scaled[256];
    for (int i = threadIdx.x; i < kDecSlices * 2 * 8 * 32; i += blockDim.x)
        (&sb[0][0][0][0])[i] = (&g_dec.bfrag[0][0][0][0])[i];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) inv_phi_scaled[i] = g_dec.inv_phi_scaled[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t ngroups = (nb + 15) / 16;
    for (int64_t grp = (int64_t)blockIdx.x * 4 + warp; grp < ngroups; grp += (int64_t)gridDim.x * 4) {
        const int64_t bA = grp * 16 + g, bB = bA + 8;
        const bool vA = bA < nb, vB = bB < nb;
        const int8_t *cA = code + bA * kKeep, *cB = code + bB * kKeep;
        uint32_t a0[4], a1[4];
        a0[0] = code_pair(cA, 2 * t, vA);
        a0[1] = code_pair(cB, 2 * t, vB);
        a0[2] = code_pair(cA, 2 * t + 8, vA);
        a0[3] = code_pair(cB, 2 * t + 8, vB);
        a1[0] = code_pair(cA, 16 + 2 * t, vA);
        a1[1] = code_pair(cB, 16 + 2 * t, vB);
        a1[2] = code_pair(cA, 24 + 2 * t, vA);
        a1[3] = code_pair(cB, 24 + 2 * t, vB);
        // Per block (h = 0: bA, 1: bB): base f, scale (s/phi) 2^E, output row
        // pointer and the logical-shape flags of a partial block.
        double fb[2], ts[2];
        double *pb[2];
        bool inside[2], c0in[2], c1in[2];
        int64_t r0[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t b = h ? bB : bA;
            const bool v = h ? vB : vA;
            const int64_t bi = v ? b / nbc : 0, bj = v ? b - bi * nbc : 0;
            fb[h] = v ? __ldg(f + b) : 0.0;
            ts[h] = v ? __ldg(s + b) * inv_phi_scaled[__ldg(phi + b)] : 0.0;  // (s / phi) 2^E
            pb[h] = A + (bi * 8) * lda + bj * 8 + 2 * t;
            r0[h] = bi * 8;
            inside[h] = bi * 8 + 8 <= rows && bj * 8 + 8 <= cols;
            c0in[h] = bj * 8 + 2 * t < cols;
            c1in[h] = bj * 8 + 2 * t + 1 < cols;
        }
        // One output row nt of every block at a time: the five slice products
        // (exact fp32 integers) are assembled and stored at once.
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            int y[kDecSlices][4];
#pragma unroll
            for (int sl = 0; sl < kDecSlices; ++sl) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_f16(c, a0, sb[sl][0][nt][lane]);
                mma_f16(c, a1, sb[sl][1][nt][lane]);
                // c + 1.5 2^23 holds the integer c in its low bits (|c| < 2^22), two at a time
                const float2 r01 = __fadd2_rn(make_float2(c[0], c[1]), make_float2(12582912.0f, 12582912.0f));
                const float2 r23 = __fadd2_rn(make_float2(c[2], c[3]), make_float2(12582912.0f, 12582912.0f));
                y[sl][0] = __float_as_int(r01.x) - 0x4B400000;
                y[sl][1] = __float_as_int(r01.y) - 0x4B400000;
                y[sl][2] = __float_as_int(r23.x) - 0x4B400000;
                y[sl][3] = __float_as_int(r23.y) - 0x4B400000;
            }
            long long acc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                acc[q] = (long long)y[0][q] * (1ll << (3 * kDecDigitBits)) +
                         (long long)y[1][q] * (1ll << (2 * kDecDigitBits)) +
                         (long long)y[2][q] * (1ll << kDecDigitBits) + y[3][q];

            }
            // c0, c1: block bA, row nt, columns 2t, 2t+1; c2, c3: block bB.
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!(h ? vB : vA)) continue;
                // M00 = f by definition (row 0 of G is zero), also when s is not finite
                const double o0 = (nt == 0 && t == 0) ? fb[h] : fma(ts[h], dec_to_double(acc[2 * h]), fb[h]);
                const double o1 = fma(ts[h], dec_to_double(acc[2 * h + 1]), fb[h]);
                if (kSlices) {
                    const int64_t b = h ? bB : bA, bi = b / nbc, bj = b - bi * nbc;
                    __nv_bfloat16 *q = Sl + (bi * 8 + nt) * 3 * kp + bj * 8 + 2 * t;
                    __nv_bfloat16 x1, x2, x3, y1, y2, y3;
                    split3(o0, x1, x2, x3);
                    split3(o1, y1, y2, y3);
                    *reinterpret_cast<__nv_bfloat162 *>(q) = __halves2bfloat162(x1, y1);
                    *reinterpret_cast<__nv_bfloat162 *>(q + kp) = __halves2bfloat162(x2, y2);
                    *reinterpret_cast<__nv_bfloat162 *>(q + 2 * kp) = __halves2bfloat162(x3, y3);
                    continue;
                }
                double *p = pb[h] + nt * lda;
                if (inside[h]) {
                    if (kVec) {
                        *reinterpret_cast<double2 *>(p) = make_double2(o0, o1);
                    } else {
                        p[0] = o0;
                        p[1] = o1;
                    }
                } else {
                    // A partial block of a padded matrix: entries outside the
                    // logical rows x cols are skipped (cropped output) or 0.
                    const bool rin = r0[h] + nt < rows;
                    if (zero_fill) {
                        p[0] = rin && c0in[h] ? o0 : 0.0;
                        p[1] = rin && c1in[h] ? o1 : 0.0;
                    } else {
                        if (rin && c0in[h]) p[0] = o0;
                        if (rin && c1in[h]) p[1] = o1;
                    }
                }
            }
        }
    }
}

// The once-per-device copy of the decompression constants (shared by both
// launchers).
static DeviceTable &dec_table()
{
    static DeviceTable t;
    return t;
}

static bool vec_ok(const void *p, int64_t ld) { return ((uintptr_t)p % 16 == 0) && (ld % 2 == 0); }

int launch_decompress(const blaz_cmat *a, double *A, int64_t lda, cudaStream_t st, int64_t rows, int64_t cols,
                      bool zero_fill)
{
    const int64_t nbc = a->cols / 8, nb = (a->rows / 8) * nbc;
    if (nb == 0) return BLAZ_OK;
    if (rows < 0) rows = a->rows;
    if (cols < 0) cols = a->cols;
    const int threads = 128;
    // One resident wave of CTAs (each first stages 20 KB of B fragments in
    // shared memory), striding over groups of 16 blocks.
    static const int occ = [] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_decompress<true>, 128, 0) != cudaSuccess) {
            (void)cudaGetLastError();
            n = 4;
        }
        return n > 0 ? n : 1;
    }();
    int64_t want = ((nb + 15) / 16 + 3) / 4;
    const int64_t cap = (int64_t)num_sms() * occ;
    const int grid = (int)std::max<int64_t>(1, std::min(want, cap));
    const int rc = dec_table().ensure(&g_dec, &dec_consts(), sizeof(DecConsts), 0, st);
    if (rc) return rc;
    if (vec_ok(A, lda))
        k_decompress<true><<<grid, threads, 0, st>>>(a->f, a->s, a->phi, a->code, nbc, nb, A, lda, rows, cols,
                                                     zero_fill);
    else
        k_decompress<false><<<grid, threads, 0, st>>>(a->f, a->s, a->phi, a->code, nbc, nb, A, lda, rows, cols,
                                                      zero_fill);
    return launch_status();
}

// The three bf16 slices of A_hat (a: full blocks, n = a->rows, k = a->cols)
// into Sl = [A1 A2 A3] (n x 3kp), columns k..kp-1 of each slice zeroed.
int launch_decompress_slices(const blaz_cmat *a, void *Sl, int64_t kp, cudaStream_t st)
{
    const int64_t nbc = a->cols / 8, nb = (a->rows / 8) * nbc, k = a->cols;
    if (nb == 0) return BLAZ_OK;
    __nv_bfloat16 *S = (__nv_bfloat16 *)Sl;
    if (kp > k) {
        // the padding columns of the 3 n rows of kp elements
        cudaError_t e = cudaMemset2DAsync(S + k, (size_t)kp * 2, 0, (size_t)(kp - k) * 2, (size_t)(3 * a->rows), st);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    static const int occ = [] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_decompress<true, true>, 128, 0) != cudaSuccess) {
            (void)cudaGetLastError();
            n = 4;
        }
        return n > 0 ? n : 1;
    }();
    int64_t want = ((nb + 15) / 16 + 3) / 4;
    const int64_t cap = (int64_t)num_sms() * occ;
    const int grid = (int)std::max<int64_t>(1, std::min(want, cap));
    const int rc = dec_table().ensure(&g_dec, &dec_consts(), sizeof(DecConsts), 0, st);
    if (rc) return rc;
    k_decompress<true, true><<<grid, 128, 0, st>>>(a->f, a->s, a->phi, a->code, nbc, nb, nullptr, 0, a->rows,
                                                   a->cols, false, S, kp);
    return launch_status();
}

}  // namespace blaz
