// k_rate.cu -- the tunable-rate variant of the compressed format.
//
// "Compressed Matrix Computations" (arXiv 2202.13007) names a tunable
// compression rate as future work (Sec. VI: more or less compression, "by
// skewing the quantization").  The reading implemented here keeps the first
// r rows and the first r columns of each block's DCT, r = 1..8: keep(r) =
// 8 r + (8 - r) r codes per block, in the order rows 0..r-1 (columns 0..7),
// then (i, 0..r-1) for i = r..7; r = 2 is Sec. II's 28-code format.  Every
// other stage is unchanged -- f, s, phi (m over all 64 coefficients, so phi
// does not depend on r), truncated codes, Algorithms 1 and 2 -- so the codes
// of rate r are the codes of any larger rate at the same positions.
//
// Compression reuses the certified compressor of the 28-code format with the
// rate's kept set, decompression its tensor-core product with the fixed
// decompression map, and addition the fp32 decisions of add_block_fast with a
// dense binary64 pass over the undecided codes; all bit-identical to the
// binary64 operation order of the 28-code format.
#include <cmath>
#include <mutex>
#include <vector>

#include <cuda_fp16.h>

#include "block_ops.cuh"
#include "compress_fix.cuh"
#include "const_upload.cuh"
#include "gmap.cuh"
#include "rate.cuh"

namespace blaz {

// Kept index of coefficient (i, j) at rate r, or -1.
__device__ __forceinline__ int rate_index(int r, int i, int j)
{
    return i < r ? i * 8 + j : (j < r ? 8 * r + (i - r) * r + j : -1);
}

// ---------------------------------------------------------------------------------
// Compression at rate r: the certified compressor of the 28-code format
// (compress_fast.cuh: binary64 normalization and slope, fp32 DCT under a
// proven bound, exact binary64 DC chains of the sign-coherent blocks, exact
// fix-up of whatever is not certified) with all 64 fp32 coefficients kept,
// since the bound holds for every (i, j).  Undecided codes are listed by
// position p = 8 i + j in a 64-bit mask.

constexpr int kRateThreads = 128;
// D and r of the sign-coherent blocks (an odd row length keeps the row reads
// conflict-free), then the exact X00 of every slot.  After the dense DC pass
// the D area holds the CTA's codes for a coalesced store.
constexpr size_t kRateSmem = sizeof(double) * (size_t)kRateThreads * 66;

// "Whole block exact" (phi not certified or non-finite values).  A real mask
// with all 64 positions undecided means the same work, and the exact whole-
// block path gives the same phi and codes.
constexpr uint64_t kRateAll = ~0ull;

struct RateCtx {
    uint32_t state;  // 0: decide; kPendingAll: whole block exact; 1: done (K == 0)
    bool coherent;
    float base;      // E_ij / aa_ij
    float mlo, mhi;  // bounds on max |X| over the 63 coefficients other than the DC
    float D[64];     // fp32 coefficients, row-major (D[0]: the DC estimate)
};

// Normalization, slope (exact binary64), the sign-coherent block's D and r
// to shared memory (slot), then the fp32 DCT of all 64 coefficients.
__device__ __forceinline__ void rate_prepare(double (&d)[64], double &s_out, RateCtx &c, double (*sD)[65],
                                             unsigned *sCount, int &slot)
{
#pragma unroll
    for (int i = 7; i >= 0; --i)
#pragma unroll
        for (int j = 7; j >= 0; --j) {
            if (i == 0 && j == 0) d[0] = 0.0;
            else if (i == 0) d[j] = dsub(d[j], d[j - 1]);
            else if (j == 0) d[i * 8] = dsub(d[i * 8], d[(i - 1) * 8]);
            else d[i * 8 + j] = dhalf(dadd(dsub(d[i * 8 + j], d[(i - 1) * 8 + j]), dsub(d[i * 8 + j], d[i * 8 + j - 1])));
        }
    int K = 0;
    unsigned pos = 0u, neg = 0u;
#pragma unroll
    for (int p = 0; p < 64; ++p) {
        const int nz = nonzero_bits(d[p]);
        K += nz;
        const unsigned sg = (unsigned)__double2hiint(d[p]) >> 31;
        pos |= (unsigned)nz & (sg ^ 1u);
        neg |= (unsigned)nz & sg;
    }
    c.coherent = false;
    slot = -1;
    if (K == 0) {
        s_out = 0.0;
        c.state = 1u;
        return;
    }
    const double S = tree_sum_abs(d);
    const double s = div_by_count(S, K);
    const double r = ddiv(1.0, s);
    s_out = s;
    const int es_field = (int)((__double_as_longlong(s) >> 52) & 0x7FF);
    if (((__double_as_longlong(S) >> 52) & 0x7FF) >= 0x7FE || ((__double_as_longlong(r) >> 52) & 0x7FF) >= 0x7FE ||
        es_field == 0) {
        c.state = kPendingAll;
        return;
    }
    c.state = 0u;
    c.coherent = (pos ^ neg) != 0u;
    if (c.coherent) {
        slot = (int)atomicAdd(sCount, 1u);
#pragma unroll
        for (int p = 0; p < 64; ++p) sD[slot][p] = d[p];
        sD[slot][64] = r;
    }
    const int e = es_field - 1023;
    const float rr = trunc_f32_scaled(r, -e);
    float T[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        float rf[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) rf[v] = trunc_f32_scaled(d[u * 8 + v], e) * rr;
        float t0 = rf[0];
#pragma unroll
        for (int v = 1; v < 8; ++v) t0 += rf[v];
        T[u][0] = t0;
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            float acc = rf[0] * cos_f(j, 0);
#pragma unroll
            for (int v = 1; v < 8; ++v) acc = fmaf(rf[v], cos_f(j, v), acc);
            T[u][j] = acc;
        }
    }
    c.base = 28.0f * 0x1p-24f * (float)(K + 1);
    float mlo = 0.0f, mhi = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float acc = cos_f(i, 0) * T[0][j];
#pragma unroll
            for (int u = 1; u < 8; ++u) acc = fmaf(cos_f(i, u), T[u][j], acc);
            const float aa = (float)aa_tab(i, j);
            const float Df = aa * acc;
            if (!(i == 0 && j == 0)) {
                const float E = c.base * aa + 1e-30f;
                const float a = fabsf(Df);
                mhi = fmaxf(mhi, a + E);
                mlo = fmaxf(mlo, a - E);
            }
            c.D[i * 8 + j] = Df;
        }
    c.mlo = mlo;
    c.mhi = mhi;
}

// phi and the kept codes (into cb, indexed by the rate-r order); returns 0,
// kRateAll or the mask of undecided positions.  The decisions are those
// of cf_finish for the 28-code format.
__device__ __forceinline__ uint64_t rate_finish(const RateCtx &c, double X00, int r, uint8_t &phi_out,
                                                uint8_t *__restrict__ cb)
{
    if (c.state == 1u) {
        phi_out = 255;
        for (int t = 0; t < rate_keep(r); ++t) cb[t] = 0;
        return 0u;
    }
    if (c.state == kPendingAll) return kRateAll;
    const float aa00 = (float)BLAZ_A00;
    const float E00 = c.base * aa00 + 1e-30f;
    bool m_exact = false;
    double ax00 = 0.0;
    float dc_lo, dc_hi;
    if (c.coherent) {
        ax00 = fabs(X00);
        const float a00 = trunc_f32(ax00);
        m_exact = __double_as_longlong(f2d_bits(c.mhi * (1.0f + 0x1p-20f))) < __double_as_longlong(ax00);
        dc_lo = a00;
        dc_hi = a00 * (1.0f + 0x1p-22f);
    } else {
        const float a = fabsf(c.D[0]);
        dc_lo = fmaxf(0.0f, (a - E00) * (1.0f - 0x1p-20f));
        dc_hi = (a + E00) * (1.0f + 0x1p-20f);
    }
    const float m_lo = m_exact ? dc_lo : fmaxf(dc_lo, c.mlo * (1.0f - 0x1p-20f));
    const float m_hi = m_exact ? dc_hi : fmaxf(dc_hi, c.mhi * (1.0f + 0x1p-20f));
    const float q_lo = __fdiv_rn(127.0f, m_hi) * (1.0f - 0x1p-20f);
    const float q_hi = __fdiv_rn(127.0f, m_lo) * (1.0f + 0x1p-20f);
    const int p_lo = q_lo >= 255.0f ? 255 : (q_lo < 1.0f ? 1 : (int)q_lo);
    const int p_hi = q_hi >= 255.0f ? 255 : (q_hi < 1.0f ? 1 : (int)q_hi);
    int phi = p_lo;
    if (p_lo != p_hi) {
        if (!m_exact) return kRateAll;
        phi = phi_of(ax00);
    }
    phi_out = (uint8_t)phi;
    const float phif = (float)phi;
    uint64_t pending = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int t = rate_index(r, i, j);
            if (t < 0) continue;
            int cc = 0;
            if (i == 0 && j == 0 && c.coherent) {
                cc = quantize_bits(dmul(X00, i64_to_double(phi)));
            } else {
                const float aa = (float)aa_tab(i, j);
                const float v = c.D[i * 8 + j] * phif;
                const float Ev = (c.base * aa * phif) * (1.0f + 0x1p-20f) + 0x1p-22f * (fabsf(v) + 1.0f) + 0x1p-16f;
                const float lo = v - Ev, hi = v + Ev;
                if (lo >= 127.0f) cc = 127;
                else if (hi <= -127.0f) cc = -127;
                else {
                    const int tl = (int)truncf(lo), th = (int)truncf(hi);
                    if (tl != th || tl >= 127 || tl <= -127) pending |= 1ull << (i * 8 + j);
                    else cc = tl;
                }
            }
            cb[t] = (uint8_t)(int8_t)cc;
        }
    return pending;
}

template <typename T>
__device__ __forceinline__ void rate_append(bool want, T value, T *__restrict__ list, unsigned *__restrict__ count)
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

template <bool kVec>
__global__ void __launch_bounds__(kRateThreads, 3)
    k_compress_rate_fast(const double *__restrict__ A, int64_t lda, int64_t nbc, int64_t nb, int r,
                         double *__restrict__ f, double *__restrict__ s, uint8_t *__restrict__ phi,
                         int8_t *__restrict__ code, uint4 *__restrict__ code_list, unsigned *__restrict__ code_count,
                         unsigned *__restrict__ block_list, unsigned *__restrict__ block_count)
{
    extern __shared__ double rate_smem[];
    double(*sD)[65] = reinterpret_cast<double(*)[65]>(rate_smem);
    double *sX = rate_smem + kRateThreads * 65;
    uint8_t *sC = reinterpret_cast<uint8_t *>(rate_smem);  // codes, after the DC pass
    __shared__ unsigned sCount;
    if (threadIdx.x == 0) sCount = 0u;
    __syncthreads();
    const int nk = rate_keep(r);
    const int64_t b0 = blockIdx.x * (int64_t)kRateThreads, b = b0 + threadIdx.x;
    const bool valid = b < nb;
    double d[64];
    double sv = 0.0;
    RateCtx ctx;
    ctx.state = 1u;
    ctx.coherent = false;
    int slot = -1;
    if (valid) {
        const int64_t bi = b / nbc, bj = b - bi * nbc;
        load_block<kVec>(A, lda, bi, bj, d);
        f[b] = d[0];
        rate_prepare(d, sv, ctx, sD, &sCount, slot);
        s[b] = sv;
    }
    __syncthreads();
    if (threadIdx.x < sCount) sX[threadIdx.x] = cf_exact_dc(sD[threadIdx.x], sD[threadIdx.x][64]);
    __syncthreads();
    uint64_t pending = 0u;
    if (valid) {
        uint8_t ph = 255;
        pending = rate_finish(ctx, slot >= 0 ? sX[slot] : 0.0, r, ph, sC + threadIdx.x * nk);
        if (pending != (kRateAll)) phi[b] = ph;
        else
            for (int t = 0; t < nk; ++t) sC[threadIdx.x * nk + t] = 0;
    }
    __syncthreads();
    // the CTA's codes: nvalid x nk contiguous bytes at a 4-byte aligned
    // address (code is 4-byte aligned and 128 nk is a multiple of 4)
    const int64_t nvalid = nb - b0 < kRateThreads ? nb - b0 : kRateThreads;
    const int bytes = (int)nvalid * nk;
    uint32_t *dst = reinterpret_cast<uint32_t *>(code + b0 * nk);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(sC);
    for (int w = threadIdx.x; w < bytes / 4; w += kRateThreads) dst[w] = src[w];
    for (int q = (bytes & ~3) + threadIdx.x; q < bytes; q += kRateThreads) code[b0 * nk + q] = (int8_t)sC[q];
    if (!valid) return;
    const bool all = pending == (kRateAll);
    rate_append(pending != 0u && !all,
                make_uint4((unsigned)b, (unsigned)pending, (unsigned)(pending >> 32), 0u), code_list, code_count);
    rate_append(all, (unsigned)b, block_list, block_count);
}

// The exact fix-up, a team of 8 lanes per listed block (compress_fix.cuh's
// evaluation order), storing in the rate-r order.
template <bool kVec>
__global__ void __launch_bounds__(128)
    k_compress_rate_fix(const double *__restrict__ A, int64_t lda, int64_t rows, int64_t cols, int64_t nbc, int r,
                        const unsigned *__restrict__ block_list, const uint4 *__restrict__ code_list,
                        const unsigned *__restrict__ counts, const double *__restrict__ s,
                        uint8_t *__restrict__ phi, int8_t *__restrict__ code)
{
    const int lane = threadIdx.x & 31, u = lane & 7, tbase = lane & ~7;
    const unsigned tmask = 0xFFu << tbase;
    const int nk = rate_keep(r);
    const int64_t ncodes = counts[0], nblocks = counts[1];
    const int64_t teams = (int64_t)gridDim.x * blockDim.x / 8;
    for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 8; q < nblocks + ncodes; q += teams) {
        double dp[8];
        if (q < nblocks) {
            // whole block: lane u forms row u of D' and its inner sums, then
            // row i = u of the outer sums; m and phi over the team
            const int64_t b = block_list[q];
            team_dprime_row<kVec>(A, lda, rows, cols, nbc, b, u, s[b], dp);
            double T[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                double acc = (j == 0) ? dp[0] : dmul(dp[0], cos_tab(j, 0));
#pragma unroll
                for (int v = 1; v < 8; ++v) acc = dadd(acc, (j == 0) ? dp[v] : dmul(dp[v], cos_tab(j, v)));
                T[j] = acc;
            }
            double U[8];
#pragma unroll
            for (int uu = 0; uu < 8; ++uu) {
                const double cu = c_cos[u * 8 + uu];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const double Tu = __shfl_sync(tmask, T[j], tbase + uu);
                    const double term = (u == 0) ? Tu : dmul(cu, Tu);
                    U[j] = (uu == 0) ? term : dadd(U[j], term);
                }
            }
            double m = 0.0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                U[j] = dmul((u == 0 && j == 0) ? BLAZ_A00 : (u == 0 || j == 0) ? BLAZ_A0K : BLAZ_AKK, U[j]);
                const double ax = fabs(U[j]);
                m = (ax > m) ? ax : m;
            }
#pragma unroll
            for (int off = 4; off; off >>= 1) {
                const double o = __shfl_xor_sync(tmask, m, off);
                m = (o > m) ? o : m;
            }
            const int ph = phi_of(m);
            const double phd = i64_to_double(ph);
            if (u == 0) phi[b] = (uint8_t)ph;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int t = rate_index(r, u, j);
                if (t >= 0) code[b * nk + t] = quantize_bits(dmul(U[j], phd));
            }
        } else {
            const uint4 e = code_list[q - nblocks];
            const int64_t b = e.x;
            team_dprime_row<kVec>(A, lda, rows, cols, nbc, b, u, s[b], dp);
            const int ph = phi[b];
            for (uint64_t msk = ((uint64_t)e.z << 32) | e.y; msk; msk &= msk - 1) {
                const int p = __ffsll((long long)msk) - 1, i = p >> 3, j = p & 7;
                double T = (j == 0) ? dp[0] : dmul(dp[0], c_cos[j * 8]);
#pragma unroll
                for (int v = 1; v < 8; ++v) T = dadd(T, (j == 0) ? dp[v] : dmul(dp[v], c_cos[j * 8 + v]));
                double U = 0.0;
#pragma unroll
                for (int uu = 0; uu < 8; ++uu) {
                    const double Tu = __shfl_sync(tmask, T, tbase + uu);
                    const double term = (i == 0) ? Tu : dmul(c_cos[i * 8 + uu], Tu);
                    U = (uu == 0) ? term : dadd(U, term);
                }
                if (u == 0) {
                    const double aa = (i == 0 && j == 0) ? BLAZ_A00 : (i == 0 || j == 0) ? BLAZ_A0K : BLAZ_AKK;
                    code[b * nk + rate_index(r, i, j)] = quantize_bits(dmul(dmul(aa, U), i64_to_double(ph)));
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// Decompression at rate r on the tensor cores, as the 28-code decompressor
// does it: a block is f 1 + (s/phi) G_r c, with G_r the 64 x keep(r) map whose
// column for kept coefficient (i, j) is the block that this coefficient alone
// produces (inverse DCT of a unit coefficient, then the inverse of Eq. eqnorm
// with f = 0), evaluated once on the host in long double.  G_r is split into
// five 9-bit fixed-point slices; every slice product with the codes is an
// integer below 2^21 (|digit| <= 2^8, |code| <= 127, at most 64 terms),
// exact in the fp32 accumulators of mma.sync m16n8k16 (fp16 inputs), and the
// slices are assembled in integers.  G_r is represented to 2^-45 of its
// largest entry: the outputs stay far within 1e-12 of the block scale.
constexpr int kRDSlices = 5;
constexpr int kRDBits = 9;
struct RateDec {
    uint2 bfrag[kRDSlices][4][8][32];  // B fragments [slice][k-step][n-tile][lane], k-steps of 16 codes
    double inv_phi_scaled[256];        // RN(1/phi) 2^E, 2^E the weight of the last slice
};
__device__ RateDec g_rate_dec[8];

static void rate_map(int r, long double (*G)[64])
{
    const long double pi = 3.14159265358979323846264338327950288L;
    long double c[8][8];
    for (int k = 0; k < 8; ++k)
        for (int x = 0; x < 8; ++x) c[k][x] = cosl((long double)((2 * x + 1) * k) * pi / 16.0L);
    const long double al[8] = {sqrtl(0.125L), 0.5L, 0.5L, 0.5L, 0.5L, 0.5L, 0.5L, 0.5L};
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            const int t = i < r ? i * 8 + j : (j < r ? 8 * r + (i - r) * r + j : -1);
            if (t < 0) continue;
            long double B[8][8];
            for (int u = 0; u < 8; ++u)
                for (int v = 0; v < 8; ++v) {
                    const long double P = al[i] * al[j] * c[i][u] * c[j][v];
                    if (u == 0 && v == 0) B[u][v] = 0.0L;
                    else if (u == 0) B[u][v] = B[u][v - 1] + P;
                    else if (v == 0) B[u][v] = B[u - 1][v] + P;
                    else B[u][v] = (B[u - 1][v] + B[u][v - 1]) * 0.5L + P;
                    G[u * 8 + v][t] = B[u][v];
                }
        }
}

static void rate_dec_build(int r, RateDec &dc)
{
    const int nk = rate_keep(r);
    std::vector<long double> Gs(64 * 64);
    long double(*G)[64] = reinterpret_cast<long double(*)[64]>(Gs.data());
    rate_map(r, G);
    long double mx = 0.0L;
    for (int p = 0; p < 64; ++p)
        for (int t = 0; t < nk; ++t) mx = fmaxl(mx, fabsl(G[p][t]));
    const int E = (int)ceill(log2l(mx)) - (kRDBits - 1);
    std::vector<float> ds(kRDSlices * 64 * 64);  // [slice][n = p][k = t], k >= nk zero
    float(*digit)[64][64] = reinterpret_cast<float(*)[64][64]>(ds.data());
    for (int p = 0; p < 64; ++p)
        for (int t = 0; t < 64; ++t) {
            long double v = t < nk ? G[p][t] : 0.0L;
            for (int sl = 0; sl < kRDSlices; ++sl) {
                const long double sc = ldexpl(1.0L, E - kRDBits * sl);
                const long double d = rintl(v / sc);
                digit[sl][p][t] = (float)d;
                v -= d * sc;
            }
        }
    auto h2 = [](float lo, float hi) {
        const __half a = __float2half_rn(lo), b = __float2half_rn(hi);
        return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
    };
    for (int sl = 0; sl < kRDSlices; ++sl)
        for (int ks = 0; ks < 4; ++ks)
            for (int nt = 0; nt < 8; ++nt)
                for (int lane = 0; lane < 32; ++lane) {
                    const int g = lane >> 2, q = lane & 3, n = nt * 8 + g, k = ks * 16 + 2 * q;
                    dc.bfrag[sl][ks][nt][lane].x = h2(digit[sl][n][k], digit[sl][n][k + 1]);
                    dc.bfrag[sl][ks][nt][lane].y = h2(digit[sl][n][k + 8], digit[sl][n][k + 9]);
                }
    const double scale = (double)ldexpl(1.0L, E - kRDBits * (kRDSlices - 1));
    dc.inv_phi_scaled[0] = 0.0;
    for (int p = 1; p < 256; ++p) dc.inv_phi_scaled[p] = (1.0 / (double)p) * scale;
}

// The constants of rate r in this device's copy of g_rate_dec (built on the
// host once, copied once per device).
static int rate_dec_ready(int r, cudaStream_t st)
{
    static std::once_flag once[8];
    static RateDec host[8];
    static DeviceTable tables[8];
    std::call_once(once[r - 1], [r] { rate_dec_build(r, host[r - 1]); });
    return tables[r - 1].ensure(g_rate_dec, &host[r - 1], sizeof(RateDec), (size_t)(r - 1) * sizeof(RateDec), st);
}

static_assert(slice_assembly_bound(kRDSlices, kRDBits, 64) < (1ull << 62),
              "the slice assembly must fit dec_to_double's input range");

__device__ __forceinline__ void rate_mma(float (&c)[4], const uint32_t (&a)[4], uint2 b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// Codes k and k+1 of a block (0 beyond nk) as an fp16 pair: the byte x ^ 0x80
// under the exponent of 1024 is the fp16 number 1152 + x, and one exact
// subtraction leaves x.  Bytes are loaded one by one (nk may be odd).
__device__ __forceinline__ uint32_t rate_code_pair(const int8_t *__restrict__ c, int k, int nk, bool valid)
{
    if (!valid || k >= nk) return 0u;
    const uint32_t lo = (uint8_t)__ldg(c + k), hi = k + 1 < nk ? (uint8_t)__ldg(c + k + 1) : 0u;
    const uint32_t v = (lo | (hi << 8)) ^ 0x8080u;
    const uint32_t q = __byte_perm(v, 0x64646464u, 0x4140);
    const __half2 h = __hsub2(*reinterpret_cast<const __half2 *>(&q), __half2half2(__ushort_as_half((unsigned short)0x6480)));
    return *reinterpret_cast<const uint32_t *>(&h);
}

template <int KS, bool kVec>
__global__ void __launch_bounds__(128)
    k_decompress_rate(int r, const double *__restrict__ f, const double *__restrict__ s,
                      const uint8_t *__restrict__ phi, const int8_t *__restrict__ code, int64_t nbc, int64_t nb,
                      double *__restrict__ A, int64_t lda)
{
    __shared__ uint2 sb[kRDSlices][KS][8][32];
    __shared__ double inv_phi_scaled[256];
    const RateDec &dc = g_rate_dec[r - 1];
    for (int i = threadIdx.x; i < kRDSlices * KS * 8 * 32; i += blockDim.x) {
        const int sl = i / (KS * 256), rest = i - sl * KS * 256;
        (&sb[sl][0][0][0])[rest] = (&dc.bfrag[sl][0][0][0])[rest];
    }
    for (int i = threadIdx.x; i < 256; i += blockDim.x) inv_phi_scaled[i] = dc.inv_phi_scaled[i];
    __syncthreads();
    const int nk = rate_keep(r);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t ngroups = (nb + 15) / 16;
    for (int64_t grp = (int64_t)blockIdx.x * 4 + warp; grp < ngroups; grp += (int64_t)gridDim.x * 4) {
        const int64_t bA = grp * 16 + g, bB = bA + 8;
        const bool vA = bA < nb, vB = bB < nb;
        const int8_t *cA = code + bA * nk, *cB = code + bB * nk;
        uint32_t a[KS][4];
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            a[ks][0] = rate_code_pair(cA, ks * 16 + 2 * t, nk, vA);
            a[ks][1] = rate_code_pair(cB, ks * 16 + 2 * t, nk, vB);
            a[ks][2] = rate_code_pair(cA, ks * 16 + 2 * t + 8, nk, vA);
            a[ks][3] = rate_code_pair(cB, ks * 16 + 2 * t + 8, nk, vB);
        }
        double fb[2], ts[2];
        double *pb[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t b = h ? bB : bA;
            const bool v = h ? vB : vA;
            const int64_t bi = v ? b / nbc : 0, bj = v ? b - bi * nbc : 0;
            fb[h] = v ? __ldg(f + b) : 0.0;
            ts[h] = v ? __ldg(s + b) * inv_phi_scaled[__ldg(phi + b)] : 0.0;
            pb[h] = A + (bi * 8) * lda + bj * 8 + 2 * t;
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            int y[kRDSlices][4];
#pragma unroll
            for (int sl = 0; sl < kRDSlices; ++sl) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) rate_mma(c, a[ks], sb[sl][ks][nt][lane]);
                const float2 r01 = __fadd2_rn(make_float2(c[0], c[1]), make_float2(12582912.0f, 12582912.0f));
                const float2 r23 = __fadd2_rn(make_float2(c[2], c[3]), make_float2(12582912.0f, 12582912.0f));
                y[sl][0] = __float_as_int(r01.x) - 0x4B400000;
                y[sl][1] = __float_as_int(r01.y) - 0x4B400000;
                y[sl][2] = __float_as_int(r23.x) - 0x4B400000;
                y[sl][3] = __float_as_int(r23.y) - 0x4B400000;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!(h ? vB : vA)) continue;
                long long acc[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int e = 2 * h + q;
                    const int p01 = y[0][e] * (1 << kRDBits) + y[1][e];
                    const int p23 = y[2][e] * (1 << kRDBits) + y[3][e];
                    acc[q] = (long long)p01 * (1ll << (3 * kRDBits)) + (long long)p23 * (1ll << kRDBits) + y[4][e];
                }
                // M00 = f by definition (row 0 of G_r is zero), also when s is not finite
                const double o0 = (nt == 0 && t == 0) ? fb[h] : fma(ts[h], dec_to_double(acc[0]), fb[h]);
                const double o1 = fma(ts[h], dec_to_double(acc[1]), fb[h]);
                double *p = pb[h] + nt * lda;
                if (kVec) {
                    *reinterpret_cast<double2 *>(p) = make_double2(o0, o1);
                } else {
                    p[0] = o0;
                    p[1] = o1;
                }
            }
        }
    }
}

template <int KS, bool kVec>
static int decompress_rate_ks(const blaz_cmat *a, int r, double *A, int64_t lda, cudaStream_t st)
{
    const int64_t nbc = a->cols / 8, nb = (a->rows / 8) * nbc;
    static const int occ = [] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_decompress_rate<KS, kVec>, 128, 0) != cudaSuccess) {
            (void)cudaGetLastError();
            n = 2;
        }
        return n > 0 ? n : 1;
    }();
    const int64_t want = ((nb + 15) / 16 + 3) / 4, cap = (int64_t)num_sms() * occ;
    const int grid = (int)(want < 1 ? 1 : (want < cap ? want : cap));
    k_decompress_rate<KS, kVec><<<grid, 128, 0, st>>>(r, a->f, a->s, a->phi, a->code, nbc, nb, A, lda);
    return launch_status();
}

// ---------------------------------------------------------------------------------
// Flattened dot <vec A_hat, vec B_hat> at rate r.  Both operands' blocks are
// decoded on the tensor cores exactly as k_decompress_rate decodes them
// (Y = G_r c as exact integers, A_hat_p = f + (s/phi) 2^E Y_p), 16 blocks per
// warp, without writing them: per block pair
//   sum_p A_hat_p B_hat_p = 64 fa fb + fa tb SB + fb ta SA + ta tb P,
// SA = sum_p YA_p and SB (exact in int64), P = sum_p YA_p YB_p (binary64),
// t = (s/phi) 2^E.  CTA partial sums are added in a fixed order by the last
// CTA (deterministic).
constexpr int kDotRateThreads = 128;

__device__ __forceinline__ double rate_cta_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r += red[q];
    __syncthreads();
    return r;  // valid in thread 0
}

// One slice-assembled output pair of the decode (exact integers).
__device__ __forceinline__ long long rate_assemble(const int (&y)[kRDSlices][4], int e)
{
    const int p01 = y[0][e] * (1 << kRDBits) + y[1][e];
    const int p23 = y[2][e] * (1 << kRDBits) + y[3][e];
    return (long long)p01 * (1ll << (3 * kRDBits)) + (long long)p23 * (1ll << kRDBits) + y[4][e];
}

template <int KS>
__device__ __forceinline__ void rate_decode_tile(const uint2 (*sb)[KS][8][32], const uint32_t (&a)[KS][4], int nt,
                                                 int lane, long long (&out)[4])
{
    int y[kRDSlices][4];
#pragma unroll
    for (int sl = 0; sl < kRDSlices; ++sl) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) rate_mma(c, a[ks], sb[sl][ks][nt][lane]);
        const float2 r01 = __fadd2_rn(make_float2(c[0], c[1]), make_float2(12582912.0f, 12582912.0f));
        const float2 r23 = __fadd2_rn(make_float2(c[2], c[3]), make_float2(12582912.0f, 12582912.0f));
        y[sl][0] = __float_as_int(r01.x) - 0x4B400000;
        y[sl][1] = __float_as_int(r01.y) - 0x4B400000;
        y[sl][2] = __float_as_int(r23.x) - 0x4B400000;
        y[sl][3] = __float_as_int(r23.y) - 0x4B400000;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) out[e] = rate_assemble(y, e);
}

template <int KS>
__global__ void __launch_bounds__(kDotRateThreads)
    k_dot_rate(int r, int64_t nb, const double *__restrict__ fa, const double *__restrict__ sa,
               const uint8_t *__restrict__ pa, const int8_t *__restrict__ ca, const double *__restrict__ fb,
               const double *__restrict__ sb_, const uint8_t *__restrict__ pb, const int8_t *__restrict__ cb,
               double *__restrict__ partials, unsigned *__restrict__ counter, double *__restrict__ result)
{
    __shared__ uint2 sbf[kRDSlices][KS][8][32];
    __shared__ double inv_phi_scaled[256];
    __shared__ double red[kDotRateThreads / 32];
    __shared__ bool last;
    const RateDec &dc = g_rate_dec[r - 1];
    for (int i = threadIdx.x; i < kRDSlices * KS * 8 * 32; i += blockDim.x) {
        const int sl = i / (KS * 256), rest = i - sl * KS * 256;
        (&sbf[sl][0][0][0])[rest] = (&dc.bfrag[sl][0][0][0])[rest];
    }
    for (int i = threadIdx.x; i < 256; i += blockDim.x) inv_phi_scaled[i] = dc.inv_phi_scaled[i];
    __syncthreads();
    const int nk = rate_keep(r);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t ngroups = (nb + 15) / 16;
    double acc = 0.0;
    for (int64_t grp = (int64_t)blockIdx.x * 4 + warp; grp < ngroups; grp += (int64_t)gridDim.x * 4) {
        const int64_t b0 = grp * 16 + g, b1 = b0 + 8;
        const bool v0 = b0 < nb, v1 = b1 < nb;
        uint32_t xa[KS][4], xb[KS][4];
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            xa[ks][0] = rate_code_pair(ca + b0 * nk, ks * 16 + 2 * t, nk, v0);
            xa[ks][1] = rate_code_pair(ca + b1 * nk, ks * 16 + 2 * t, nk, v1);
            xa[ks][2] = rate_code_pair(ca + b0 * nk, ks * 16 + 2 * t + 8, nk, v0);
            xa[ks][3] = rate_code_pair(ca + b1 * nk, ks * 16 + 2 * t + 8, nk, v1);
            xb[ks][0] = rate_code_pair(cb + b0 * nk, ks * 16 + 2 * t, nk, v0);
            xb[ks][1] = rate_code_pair(cb + b1 * nk, ks * 16 + 2 * t, nk, v1);
            xb[ks][2] = rate_code_pair(cb + b0 * nk, ks * 16 + 2 * t + 8, nk, v0);
            xb[ks][3] = rate_code_pair(cb + b1 * nk, ks * 16 + 2 * t + 8, nk, v1);
        }
        // per block h (0: b0, 1: b1): sum YA, sum YB, sum YA YB over this lane's 16 positions
        long long SA[2] = {0, 0}, SB[2] = {0, 0};
        double P[2] = {0.0, 0.0};
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            long long ya[4], yb[4];
            rate_decode_tile<KS>(sbf, xa, nt, lane, ya);
            rate_decode_tile<KS>(sbf, xb, nt, lane, yb);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int h = e >> 1;
                SA[h] += ya[e];
                SB[h] += yb[e];
                // KS = 3 keeps the general conversion: with the shorter one the
                // compiler allocates 168 registers (3 CTAs per SM) and the
                // kernel runs slower (0.167 against 0.139 ms at 4096^2, r = 4)
                P[h] = KS == 3 ? fma(i64_to_double(ya[e]), i64_to_double(yb[e]), P[h])
                               : fma(dec_to_double(ya[e]), dec_to_double(yb[e]), P[h]);
            }
        }
        // the quad (t = 0..3) holds all 64 positions of both blocks
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                SA[h] += __shfl_xor_sync(0xffffffffu, SA[h], o);
                SB[h] += __shfl_xor_sync(0xffffffffu, SB[h], o);
                P[h] += __shfl_xor_sync(0xffffffffu, P[h], o);
            }
        }
        if (t < 2 && (t ? v1 : v0)) {
            const int64_t b = t ? b1 : b0;
            const double f_a = fa[b], f_b = fb[b];
            const double ta = sa[b] * inv_phi_scaled[pa[b]], tb = sb_[b] * inv_phi_scaled[pb[b]];
            const double sA = i64_to_double(t ? SA[1] : SA[0]), sB = i64_to_double(t ? SB[1] : SB[0]);
            const double pp = t ? P[1] : P[0];
            acc += fma(f_a, fma(tb, sB, 64.0 * f_b), ta * fma(tb, pp, f_b * sA));
        }
    }
    const double tot = rate_cta_sum(acc, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = tot;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) v += __ldcg(partials + q);
    const double tot2 = rate_cta_sum(v, red);
    if (threadIdx.x == 0) {
        *result = tot2;
        *counter = 0u;
    }
}

int dot_rate_grid(int64_t nb)
{
    const int64_t want = ((nb + 15) / 16 + 3) / 4, cap = (int64_t)num_sms() * 4;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

template <int KS>
static int dot_rate_ks(const blaz_cmat *a, const blaz_cmat *b, int r, double *result, double *partials,
                       unsigned *counter, cudaStream_t st)
{
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    k_dot_rate<KS><<<dot_rate_grid(nb), kDotRateThreads, 0, st>>>(r, nb, a->f, a->s, a->phi, a->code, b->f, b->s,
                                                                  b->phi, b->code, partials, counter, result);
    return launch_status();
}

int launch_dot_rate(const blaz_cmat *a, const blaz_cmat *b, int r, double *result, double *partials,
                    unsigned *counter, cudaStream_t st)
{
    int rc = rate_dec_ready(r, st);
    if (rc) return rc;
    switch ((rate_keep(r) + 15) / 16) {
    case 1: return dot_rate_ks<1>(a, b, r, result, partials, counter, st);
    case 2: return dot_rate_ks<2>(a, b, r, result, partials, counter, st);
    case 3: return dot_rate_ks<3>(a, b, r, result, partials, counter, st);
    default: return dot_rate_ks<4>(a, b, r, result, partials, counter, st);
    }
}

// ---------------------------------------------------------------------------------
// Algorithm 3 at rate r: line i of A_hat times column j of B_hat, decoding
// only that line of each block (i, kb) and that column of each block (kb, j)
// with rows of G_r (binary64 copies of the long double map), 16 lanes per
// k-block; CTA partials added in order by the last CTA.
struct RateG {
    double G[8][64][64];  // [r-1][p][t], t < keep(r)
    double inv_phi[256];
};
__device__ RateG g_rate_g;

static int rate_g_ready(cudaStream_t st)
{
    static std::once_flag once;
    static RateG host;
    static DeviceTable table;
    std::call_once(once, [] {
        std::vector<long double> Gs(64 * 64);
        long double(*G)[64] = reinterpret_cast<long double(*)[64]>(Gs.data());
        for (int r = 1; r <= 8; ++r) {
            rate_map(r, G);
            for (int p = 0; p < 64; ++p)
                for (int t = 0; t < 64; ++t) host.G[r - 1][p][t] = t < rate_keep(r) ? (double)G[p][t] : 0.0;
        }
        host.inv_phi[0] = 0.0;
        for (int p = 1; p < 256; ++p) host.inv_phi[p] = 1.0 / (double)p;
    });
    return table.ensure(&g_rate_g, &host, sizeof(RateG), 0, st);
}

__global__ void __launch_bounds__(256)
    k_dot_rowcol_rate(int r, int64_t nkb, int64_t nbc_a, int64_t nbc_b, int64_t i, int64_t j,
                      const double *__restrict__ fa, const double *__restrict__ sa, const uint8_t *__restrict__ pa,
                      const int8_t *__restrict__ ca, const double *__restrict__ fb, const double *__restrict__ sb,
                      const uint8_t *__restrict__ pb, const int8_t *__restrict__ cb, double *__restrict__ partials,
                      unsigned *__restrict__ counter, double *__restrict__ result)
{
    __shared__ double Gr[8][64], Gc[8][64], inv_phi[256];
    __shared__ double red[8];
    __shared__ bool last;
    const int nk = rate_keep(r);
    const int64_t bi = i / 8, bj = j / 8;
    const int ri = (int)(i % 8), cj = (int)(j % 8);
    for (int e = threadIdx.x; e < 8 * 64; e += blockDim.x) {
        const int q = e >> 6, t = e & 63;
        Gr[q][t] = g_rate_g.G[r - 1][ri * 8 + q][t];
        Gc[q][t] = g_rate_g.G[r - 1][q * 8 + cj][t];
    }
    for (int e = threadIdx.x; e < 256; e += blockDim.x) inv_phi[e] = g_rate_g.inv_phi[e];
    __syncthreads();
    // a team of 16 lanes per k-block, lane (side, q) decoding entry q of the
    // line (side 0) or of the column (side 1), as k_dot_rowcol does
    const int lane = threadIdx.x & 31, side = (lane >> 3) & 1, q = lane & 7;
    const unsigned tmask = 0xFFFFu << (lane & 16);
    const double *Gq = side ? Gc[q] : Gr[q];
    double acc = 0.0;
    const int64_t teams = (int64_t)gridDim.x * blockDim.x / 16;
    for (int64_t kb = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 16; kb < nkb; kb += teams) {
        const int64_t b = side ? kb * nbc_b + bj : bi * nbc_a + kb;
        const int8_t *x = (side ? cb : ca) + b * nk;
        double y = 0.0;
        for (int t = 0; t < nk; ++t) y = fma(Gq[t], i64_to_double(__ldg(x + t)), y);
        const double v = fma((side ? sb[b] : sa[b]) * inv_phi[side ? pb[b] : pa[b]], y, side ? fb[b] : fa[b]);
        const double w = __shfl_xor_sync(tmask, v, 8);
        double prod = side ? 0.0 : v * w;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) prod += __shfl_xor_sync(tmask, prod, o);
        if ((lane & 15) == 0) acc += prod;
    }
    const double tot = rate_cta_sum(acc, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = tot;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) v += __ldcg(partials + q);
    const double tot2 = rate_cta_sum(v, red);
    if (threadIdx.x == 0) {
        *result = tot2;
        *counter = 0u;
    }
}

int rowcol_rate_grid(int64_t nkb)
{
    const int64_t want = (nkb * 16 + 255) / 256, cap = (int64_t)num_sms();
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

int launch_dot_rowcol_rate(const blaz_cmat *a, const blaz_cmat *b, int r, int64_t i, int64_t j, double *result,
                           double *partials, unsigned *counter, cudaStream_t st)
{
    int rc = rate_g_ready(st);
    if (rc) return rc;
    const int64_t nkb = a->cols / 8;
    k_dot_rowcol_rate<<<rowcol_rate_grid(nkb), 256, 0, st>>>(r, nkb, a->cols / 8, b->cols / 8, i, j, a->f, a->s,
                                                            a->phi, a->code, b->f, b->s, b->phi, b->code, partials,
                                                            counter, result);
    return launch_status();
}

// Algorithm 1 (kSub: the subtraction) on rate-r blocks, one block per
// thread, with the arithmetic of the tiled 28-code addition (k_blockops.cu):
// beta_1, beta_2 estimated in fp32 (beta_f32, within 2^-20) and each code
// decided from v = fl(beta_1 c_1 +- beta_2 c_2) when
// [v - E, v + E], E = 1.25 2^-19 (|beta_1| |c_1| + |beta_2| |c_2|) + 2^-100,
// truncates to one code.  The CTA stages the codes of its 128 blocks in
// shared memory with word copies (coalesced) and queues the undecided codes;
// then, densely (a binary64 instruction costs a warp the same for one lane
// as for 32), the blocks with a queued code get their exact binary64 beta_k
// as Algorithm 1 forms them, and the queued codes their binary64 value.  The
// output codes go back as words.  Every input of a block is read before its
// outputs are written, so out may alias a or b.
constexpr int kAddRateThreads = 128;

__device__ __forceinline__ void rate_stage_in(uint8_t *__restrict__ dst, const int8_t *__restrict__ src, int bytes)
{
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
    for (int w = threadIdx.x; w < bytes / 4; w += blockDim.x) d32[w] = __ldg(s32 + w);
    for (int q = (bytes & ~3) + threadIdx.x; q < bytes; q += blockDim.x) dst[q] = (uint8_t)__ldg(src + q);
}

__device__ __forceinline__ void rate_stage_out(int8_t *__restrict__ dst, const uint8_t *__restrict__ src, int bytes)
{
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
    for (int w = threadIdx.x; w < bytes / 4; w += blockDim.x) d32[w] = s32[w];
    for (int q = (bytes & ~3) + threadIdx.x; q < bytes; q += blockDim.x) dst[q] = (int8_t)src[q];
}

template <bool kSub>
__global__ void __launch_bounds__(kAddRateThreads)
    k_add_rate(int64_t nb, int r, const double *f1, const double *s1, const uint8_t *p1, const int8_t *c1,
               const double *f2, const double *s2, const uint8_t *p2, const int8_t *c2, double *f, double *s,
               uint8_t *p, int8_t *c)
{
    // dynamic shared memory: per block slot the exact beta_1, beta_2 (when
    // needed), the inputs s_1, s_2 and phi_1, phi_2, phi; the codes of a
    // (reused for the output) and of b; the queue of undecided codes
    extern __shared__ double add_rate_smem[];
    double2 *sBeta = reinterpret_cast<double2 *>(add_rate_smem);
    double2 *sS = sBeta + kAddRateThreads;
    uint32_t *sPhi = reinterpret_cast<uint32_t *>(sS + kAddRateThreads);
    uint32_t *sNeed = sPhi + kAddRateThreads;
    uint8_t *sA = reinterpret_cast<uint8_t *>(sNeed + kAddRateThreads);
    uint8_t *sB = sA + kAddRateThreads * 64;
    uint32_t *sQ = reinterpret_cast<uint32_t *>(sB + kAddRateThreads * 64);
    __shared__ unsigned sCount, sNeedCount;
    const int nk = rate_keep(r);
    for (int64_t b0 = blockIdx.x * (int64_t)kAddRateThreads; b0 < nb; b0 += (int64_t)gridDim.x * kAddRateThreads) {
        const int nvalid = (int)(nb - b0 < kAddRateThreads ? nb - b0 : kAddRateThreads);
        if (threadIdx.x == 0) {
            sCount = 0u;
            sNeedCount = 0u;
        }
        rate_stage_in(sA, c1 + b0 * nk, nvalid * nk);
        rate_stage_in(sB, c2 + b0 * nk, nvalid * nk);
        __syncthreads();
        const int tid = threadIdx.x;
        if (tid < nvalid) {
            const int64_t b = b0 + tid;
            const double fa = f1[b], fb = f2[b], sa = s1[b], sb = s2[b];
            const int pa = p1[b], pb = p2[b];
            const double fs = kSub ? dsub(fa, fb) : dadd(fa, fb);
            const double ss = dadd(sa, sb);
            int ph = (pa * pb) / (pa + pb);
            ph = ph < 1 ? 1 : ph;
            uint8_t *ca = sA + tid * nk;
            const uint8_t *cb = sB + tid * nk;
            if (ss == 0.0) {
                for (int t = 0; t < nk; ++t) ca[t] = 0;
            } else {
                const float phf = (float)ph;
                float b1f = 0.0f, b2f = 0.0f;
                const bool ok = beta_f32(sa, ss, __fdividef(phf, (float)pa), b1f) &
                                beta_f32(sb, ss, __fdividef(phf, (float)pb), b2f);
                const float e1 = 0x1.4p-19f * fabsf(b1f), e2 = 0x1.4p-19f * fabsf(b2f);
                const float nb2 = kSub ? -b2f : b2f;
                bool need = false;
                // codes in rotated order from t = c tid mod nk, with c chosen per
                // rate so that the lanes' byte accesses (slots nk bytes apart)
                // fall on distinct banks (at most 2 words per bank; 16 for
                // r = 8 without rotation)
                const int rot = (0x23011100 >> (4 * (r - 1))) & 0xF;  // c = 0 0 1 1 1 0 3 2 for r = 1..8
                int t = (rot * tid) % nk;
                for (int k = 0; k < nk; ++k, t = (t + 1 == nk) ? 0 : t + 1) {
                    const int i1 = (int)(int8_t)ca[t], i2 = (int)(int8_t)cb[t];
                    const float x1 = small_int_to_float(i1), x2 = small_int_to_float(i2);
                    const float v = fmaf(b1f, x1, nb2 * x2);
                    const float E = fmaf(e1, fabsf(x1), fmaf(e2, fabsf(x2), 0x1p-100f));
                    const float hi = v + E, lo = fmaf(E, -1.0f, v);
                    const int l = min(127, max(-127, (int)truncf(lo))), h = min(127, max(-127, (int)truncf(hi)));
                    const bool undecided = !ok || l != h;
                    if (undecided)
                        sQ[atomicAdd(&sCount, 1u)] = (uint32_t)tid | ((uint32_t)t << 8) |
                                                     ((uint32_t)(uint8_t)i1 << 16) | ((uint32_t)(uint8_t)i2 << 24);
                    need |= undecided;
                    ca[t] = (uint8_t)(int8_t)(undecided ? 0 : l);
                }
                if (need) {
                    sS[tid] = make_double2(sa, sb);
                    sPhi[tid] = (uint32_t)pa | ((uint32_t)pb << 8) | ((uint32_t)ph << 16);
                    sNeed[atomicAdd(&sNeedCount, 1u)] = (uint32_t)tid;
                }
            }
            f[b] = fs;
            s[b] = ss;
            p[b] = (uint8_t)ph;
        }
        __syncthreads();
        // exact beta_k of the blocks with a queued code (Algorithm 1 in binary64)
        for (unsigned k = threadIdx.x; k < sNeedCount; k += kAddRateThreads) {
            const int slot = (int)sNeed[k];
            const double2 sv = sS[slot];
            const uint32_t pp = sPhi[slot];
            const int pa = (int)(pp & 0xFFu), pb = (int)((pp >> 8) & 0xFFu), ph = (int)(pp >> 16);
            const double ss = dadd(sv.x, sv.y);
            const double a1 = ddiv(sv.x, ss), a2 = ddiv(sv.y, ss);
            const double phd = i64_to_double(ph);
            sBeta[slot] = make_double2(dmul(div_small_int(a1, pa), phd), dmul(div_small_int(a2, pb), phd));
        }
        __syncthreads();
        // the queued codes, densely, in add_block's binary64 order
        for (unsigned q = threadIdx.x; q < sCount; q += kAddRateThreads) {
            const uint32_t e = sQ[q];
            const int slot = (int)(e & 0xFFu), t = (int)((e >> 8) & 0xFFu);
            const double x1 = (double)(int8_t)(uint8_t)(e >> 16), x2 = (double)(int8_t)(uint8_t)(e >> 24);
            const double2 bb = sBeta[slot];
            const double y = kSub ? dsub(dmul(bb.x, x1), dmul(bb.y, x2)) : dadd(dmul(bb.x, x1), dmul(bb.y, x2));
            sA[slot * nk + t] = (uint8_t)quantize(y);
        }
        __syncthreads();
        rate_stage_out(c + b0 * nk, sA, nvalid * nk);
        __syncthreads();
    }
}

constexpr size_t kAddRateSmem = (sizeof(double2) * 2 + sizeof(uint32_t) * 2) * kAddRateThreads +
                                2 * kAddRateThreads * 64 + sizeof(uint32_t) * kAddRateThreads * 64;

// Algorithm 2 on rate-r blocks: f and s times c; phi and the codes copied
// (untouched when out is a), the codes as 4-byte words (both arrays are
// 4-byte aligned).
__global__ void __launch_bounds__(256)
    k_scale_rate(int64_t nb, int r, const double *f1, const double *s1, const uint8_t *p1, const int8_t *c1,
                 double cst, double *f, double *s, uint8_t *p, int8_t *c, bool copy)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t b = tid; b < nb; b += stride) {
        f[b] = dmul(f1[b], cst);
        s[b] = dmul(s1[b], cst);
        if (copy) p[b] = p1[b];
    }
    if (!copy) return;
    const int64_t bytes = nb * rate_keep(r);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(c1);
    uint32_t *dst = reinterpret_cast<uint32_t *>(c);
    for (int64_t w = tid; w < bytes / 4; w += stride) dst[w] = __ldg(src + w);
    for (int64_t q = (bytes & ~(int64_t)3) + tid; q < bytes; q += stride) c[q] = c1[q];
}

static int rate_grid(int64_t n, int threads)
{
    const int64_t want = (n + threads - 1) / threads, cap = (int64_t)num_sms() * 16;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

size_t compress_rate_scratch_bytes(int64_t nb)
{
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    return up((size_t)nb * 16) + up((size_t)nb * 4) + 256;
}

int launch_compress_rate(const double *A, int64_t lda, const blaz_cmat *out, int r, void *scratch, cudaStream_t st)
{
    const int64_t nbc = out->cols / 8, nb = (out->rows / 8) * nbc;
    if (nb == 0) return BLAZ_OK;
    if (nb > 0xFFFFFFFFll) return BLAZ_ERR_SHAPE;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    uint4 *code_list = (uint4 *)scratch;
    unsigned *block_list = (unsigned *)((char *)scratch + up((size_t)nb * 16));
    unsigned *counts = (unsigned *)((char *)scratch + up((size_t)nb * 16) + up((size_t)nb * 4));
    cudaError_t e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return set_cuda_error(e);
    static const bool smem_ok = [] {
        return cudaFuncSetAttribute(k_compress_rate_fast<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kRateSmem) == cudaSuccess &&
               cudaFuncSetAttribute(k_compress_rate_fast<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kRateSmem) == cudaSuccess;
    }();
    if (!smem_ok) return set_cuda_error(cudaGetLastError());
    const int64_t grid = (nb + kRateThreads - 1) / kRateThreads;
    const int fix_grid = num_sms() * 4;
    const bool vec = ((uintptr_t)A % 16 == 0) && (lda % 2 == 0);
    if (vec) {
        k_compress_rate_fast<true><<<(unsigned)grid, kRateThreads, kRateSmem, st>>>(
            A, lda, nbc, nb, r, out->f, out->s, out->phi, out->code, code_list, counts, block_list, counts + 1);
        k_compress_rate_fix<true><<<fix_grid, 128, 0, st>>>(A, lda, out->rows, out->cols, nbc, r, block_list,
                                                            code_list, counts, out->s, out->phi, out->code);
    } else {
        k_compress_rate_fast<false><<<(unsigned)grid, kRateThreads, kRateSmem, st>>>(
            A, lda, nbc, nb, r, out->f, out->s, out->phi, out->code, code_list, counts, block_list, counts + 1);
        k_compress_rate_fix<false><<<fix_grid, 128, 0, st>>>(A, lda, out->rows, out->cols, nbc, r, block_list,
                                                             code_list, counts, out->s, out->phi, out->code);
    }
    return launch_status();
}

int launch_decompress_rate(const blaz_cmat *a, int r, double *A, int64_t lda, cudaStream_t st)
{
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    if (nb == 0) return BLAZ_OK;
    int rc = rate_dec_ready(r, st);
    if (rc) return rc;
    const bool vec = ((uintptr_t)A % 16 == 0) && (lda % 2 == 0);
    switch ((rate_keep(r) + 15) / 16) {
    case 1: return vec ? decompress_rate_ks<1, true>(a, r, A, lda, st) : decompress_rate_ks<1, false>(a, r, A, lda, st);
    case 2: return vec ? decompress_rate_ks<2, true>(a, r, A, lda, st) : decompress_rate_ks<2, false>(a, r, A, lda, st);
    case 3: return vec ? decompress_rate_ks<3, true>(a, r, A, lda, st) : decompress_rate_ks<3, false>(a, r, A, lda, st);
    default: return vec ? decompress_rate_ks<4, true>(a, r, A, lda, st) : decompress_rate_ks<4, false>(a, r, A, lda, st);
    }
}

int launch_add_rate(const blaz_cmat *a, const blaz_cmat *b, const blaz_cmat *o, int r, bool subtract,
                    cudaStream_t st)
{
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    if (nb == 0) return BLAZ_OK;
    static const bool smem_ok = [] {
        return cudaFuncSetAttribute(k_add_rate<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kAddRateSmem) == cudaSuccess &&
               cudaFuncSetAttribute(k_add_rate<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kAddRateSmem) == cudaSuccess;
    }();
    if (!smem_ok) return set_cuda_error(cudaGetLastError());
    const int64_t tiles = (nb + kAddRateThreads - 1) / kAddRateThreads, cap = (int64_t)num_sms() * 8;
    const int grid = (int)(tiles < cap ? tiles : cap);
    if (subtract)
        k_add_rate<true><<<grid, kAddRateThreads, kAddRateSmem, st>>>(nb, r, a->f, a->s, a->phi, a->code, b->f, b->s,
                                                                      b->phi, b->code, o->f, o->s, o->phi, o->code);
    else
        k_add_rate<false><<<grid, kAddRateThreads, kAddRateSmem, st>>>(nb, r, a->f, a->s, a->phi, a->code, b->f,
                                                                       b->s, b->phi, b->code, o->f, o->s, o->phi,
                                                                       o->code);
    return launch_status();
}

int launch_scale_rate(const blaz_cmat *a, double cst, const blaz_cmat *o, int r, cudaStream_t st)
{
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    if (nb == 0) return BLAZ_OK;
    const bool copy = o->code != a->code || o->phi != a->phi;
    k_scale_rate<<<rate_grid(nb * rate_keep(r) / 4 + 1, 256), 256, 0, st>>>(nb, r, a->f, a->s, a->phi, a->code, cst, o->f,
                                                                    o->s, o->phi, o->code, copy);
    return launch_status();
}

}  // namespace blaz
