// k_blockops.cu -- operations on compressed blocks without decompression:
// addition / subtraction (Algorithm 1, Eq. eq55) and multiplication by a
// constant (Algorithm 2) of "Compressed Matrix Computations" (arXiv 2202.13007).
// Bit-exact binary64 (explicit round-to-nearest intrinsics).
#include <algorithm>

#include "block_ops.cuh"
#include "tcgen05.cuh"

namespace blaz {

template <bool kSub>
__global__ void __launch_bounds__(128)
    k_add(int64_t nb, const double *__restrict__ f1, const double *__restrict__ s1, const uint8_t *__restrict__ p1,
          const int8_t *__restrict__ c1, const double *__restrict__ f2, const double *__restrict__ s2,
          const uint8_t *__restrict__ p2, const int8_t *__restrict__ c2, double *f, double *s, uint8_t *p,
          int8_t *c)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x)
        add_block_fast<kSub>(b, f1, s1, p1, c1, f2, s2, p2, c2, f, s, p, c);
}

// Algorithm 1 over tiles of kAddTile blocks with the four binary64 divisions
// taken out of the common path.  Eight compute warps (one block per thread)
// stage every input of a tile (the codes, f, s and phi of both operands)
// with asynchronous copies into shared memory, the next tile's copies in
// flight while the current one is decided (a thread's 28 codes are 7 words
// at stride 7: conflict-free), form beta_k in fp32 (beta_f32) and decide
// each code from v = fl(beta_1 c_1 +- beta_2 c_2) and the bound
//   |v - y| <= 2^-19 (|beta_1 c_1| + |beta_2 c_2|) + 2^-22 |v| + 2^-100
// (2^-20 from beta, 2^-23 from the fp32 product and fma, the binary64
// roundings of the specification far below).  With |c_k| <= 128 and
// |v| <= (|beta_1 c_1| + |beta_2 c_2|)(1 + 2^-20) the bound is at most
// 1.125 2^-12 (|beta_1| + |beta_2|) + 2^-100, so one half-width serves the
// whole block: E = 1.25 2^-12 (|beta_1| + |beta_2|) + 2^-100 (the factor
// 1.25 covers the fp32 roundings of E and of v +- E).  A code is decided
// when v - E and v + E truncate to the same int8 (saturating conversions,
// four codes per word compared at once) other than -128, the saturated
// value below quantize's -127.  f and s are two binary64 additions per
// block.  One CTA barrier per tile: the copies of the next tile go out just
// after it, into the stage every thread has finished with.
//
// A block with an undecided code, or whose beta_k has no fp32 estimate, goes
// to a per-tile list with copies of its inputs.  Undecided codes are
// structural rather than rare: equal phi and equal codes in both operands put
// y on an integer (y = c phi / phi_k in real arithmetic).  Two more warps,
// the fixers, evaluate the listed blocks in binary64 (add_block's
// arithmetic, undecided codes only; up to 32 blocks per pass of a warp,
// since a binary64 instruction costs a warp the same for one lane as for
// 32): one forms beta_1 and the other beta_2 of every listed block, so the
// division chains run on two warps at once, then each evaluates the
// undecided codes of one parity, with conversions and quantize on the
// integer pipe; they patch the tile's output codes in shared memory and
// store them with 16-byte writes, while the compute warps already decide the
// next tile: the two sides share double-buffered output tiles and lists
// through mbarriers (bounded waits; BLAZ_ERR_TIMEOUT in the status word of
// these kernels).
//
// Every input of a tile is read before any output of it is written, so out
// may alias a or b.  Requires 16-byte aligned code, f, s and phi arrays of
// both operands and an aligned output code array (the launcher checks).
constexpr int kAddTile = 256;   // blocks per tile (one per compute thread)
constexpr int kAddStages = 2;   // input stages: the tile decided and the next one
constexpr int kAddOut = 2;      // output tiles and lists shared with the fixers
constexpr int kAddCtas = 3;     // resident CTAs per SM (shared memory: 3 x 74 KB)
constexpr int kAddFixCap = kAddTile / 4;    // list entries per tile; beyond, the block's own thread fixes it

struct AddFix {
    double sa, sb, ss;      // s_1, s_2 and s = s_1 + s_2
    uint32_t wa[7], wb[7];  // the block's codes (the input stage is refilled before the fixers run)
    uint32_t undecided;     // bit 8k+q: code 4q+k (byte k of word q)
    int t, pa, pb, ph;
};

// Every input of one tile: the codes of both operands (7 words per block),
// f, s and phi of both.  16-byte aligned arrays (kAddTile a multiple of 16).
struct AddStage {
    uint32_t ca[kAddTile * 7], cb[kAddTile * 7];
    double fa[kAddTile], fb[kAddTile], sa[kAddTile], sb[kAddTile];
    uint8_t pa[kAddTile], pb[kAddTile];
};
static_assert(kAddTile % 16 == 0 && sizeof(AddStage) == 90 * kAddTile && kAddStages >= 2, "stage layout");

__device__ int g_ops_status;  // 0 or BLAZ_ERR_TIMEOUT (tiled addition)

// input stages, output tiles, lists
constexpr size_t kAddSmem =
    kAddStages * sizeof(AddStage) + kAddOut * kAddTile * 7 * 4 + kAddOut * kAddFixCap * sizeof(AddFix);

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// this thread's copies of all but the newest kAddStages - 2 groups have
// landed (the groups of the tiles ahead of the current one, committed after
// its barrier)
__device__ __forceinline__ void cp_async_wait_stage()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(kAddStages - 2) : "memory");
}

// 16-byte copies of `bytes` (a multiple of 16) by the kAddTile compute threads.
__device__ __forceinline__ void stage_copy16(void *dst, const void *src, int bytes, int t)
{
    for (int i = t; i < bytes / 16; i += kAddTile)
        cp_async16(static_cast<uint4 *>(dst) + i, static_cast<const uint4 *>(src) + i);
}

// Starts the copies of every input of one tile into a stage.  A ragged last
// tile copies words (codes), 8-byte elements (f, s) and, phi, plain bytes.
__device__ __forceinline__ void add_stage(int64_t tile, int64_t nb, const double *f1, const double *s1,
                                          const uint8_t *p1, const int8_t *c1, const double *f2, const double *s2,
                                          const uint8_t *p2, const int8_t *c2, AddStage &st, int t)
{
    const int64_t b0 = tile * kAddTile;
    const int nt = (int)(nb - b0 < kAddTile ? nb - b0 : (int64_t)kAddTile);
    if (nt == kAddTile) {
        stage_copy16(st.ca, c1 + b0 * kKeep, kAddTile * kKeep, t);
        stage_copy16(st.cb, c2 + b0 * kKeep, kAddTile * kKeep, t);
        stage_copy16(st.fa, f1 + b0, kAddTile * 8, t);
        stage_copy16(st.fb, f2 + b0, kAddTile * 8, t);
        stage_copy16(st.sa, s1 + b0, kAddTile * 8, t);
        stage_copy16(st.sb, s2 + b0, kAddTile * 8, t);
        stage_copy16(st.pa, p1 + b0, kAddTile, t);
        stage_copy16(st.pb, p2 + b0, kAddTile, t);
    } else {
        const uint32_t *ga = reinterpret_cast<const uint32_t *>(c1 + b0 * kKeep);
        const uint32_t *gb = reinterpret_cast<const uint32_t *>(c2 + b0 * kKeep);
        for (int i = t; i < nt * 7; i += kAddTile) {
            cp_async4(st.ca + i, ga + i);
            cp_async4(st.cb + i, gb + i);
        }
        if (t < nt) {
            cp_async8(st.fa + t, f1 + b0 + t);
            cp_async8(st.fb + t, f2 + b0 + t);
            cp_async8(st.sa + t, s1 + b0 + t);
            cp_async8(st.sb + t, s2 + b0 + t);
            st.pa[t] = p1[b0 + t];
            st.pb[t] = p2[b0 + t];
        }
    }
}

// binary64 Algorithm 1 for the undecided codes of one block (bit 8k+q of
// `undecided`: code k of word q), patched into its output words.
template <bool kSub>
__device__ __forceinline__ void add_fix_block(double sa, double sb, int pa, int pb, const uint32_t *wa,
                                              const uint32_t *wb, uint32_t undecided, uint32_t *wo)
{
    const double ss = dadd(sa, sb);
    int ph = (pa * pb) / (pa + pb);
    ph = ph < 1 ? 1 : ph;
    const double a1 = ddiv(sa, ss);
    const double a2 = ddiv(sb, ss);
    const double phd = i64_to_double(ph);
    const double b1 = dmul(div_small_int(a1, pa), phd);
    const double b2 = dmul(div_small_int(a2, pb), phd);
    // one pass per undecided code (the lane's set bits, lowest first)
    for (uint32_t m = undecided; m; m &= m - 1u) {
        const int bit = __ffs(m) - 1, q = bit & 7, k = bit >> 3;
        // the conversions and quantize on the integer pipe: three binary64
        // operations per code
        const double x1 = i64_to_double((int8_t)(uint8_t)(wa[q] >> (8 * k)));
        const double x2 = i64_to_double((int8_t)(uint8_t)(wb[q] >> (8 * k)));
        const double y = kSub ? dsub(dmul(b1, x1), dmul(b2, x2)) : dadd(dmul(b1, x1), dmul(b2, x2));
        reinterpret_cast<int8_t *>(wo + q)[k] = quantize_bits(y);
    }
}

// The two halves of add_fix_block for a pair of fixer warps: each forms one
// beta_k = RN(RN(RN(s_k / s) / phi_k) phi) (s and phi as the compute warps
// formed them) as add_fix_block does, so the binary64 division chains of a
// tile's list
// run on two warps (the binary64 issue rate is per warp instruction, not per
// lane: splitting lanes would not shorten the chain, splitting instructions
// does).
__device__ __forceinline__ double add_fix_beta(double sk, double ss, int pk, int ph)
{
    return dmul(div_small_int(ddiv(sk, ss), pk), i64_to_double(ph));
}

// The undecided codes 4q+k of one block with k of parity `par` (the other
// fixer warp takes the others), from beta_1 and beta_2.
template <bool kSub>
__device__ __forceinline__ void add_fix_codes(double b1, double b2, const uint32_t *wa, const uint32_t *wb,
                                              uint32_t undecided, int par, uint32_t *wo)
{
    for (uint32_t m = undecided & (par ? 0xFF00FF00u : 0x00FF00FFu); m; m &= m - 1u) {
        const int bit = __ffs(m) - 1, q = bit & 7, k = bit >> 3;
        // the conversions and quantize on the integer pipe: three binary64
        // operations per code
        const double x1 = i64_to_double((int8_t)(uint8_t)(wa[q] >> (8 * k)));
        const double x2 = i64_to_double((int8_t)(uint8_t)(wb[q] >> (8 * k)));
        const double y = kSub ? dsub(dmul(b1, x1), dmul(b2, x2)) : dadd(dmul(b1, x1), dmul(b2, x2));
        reinterpret_cast<int8_t *>(wo + q)[k] = quantize_bits(y);
    }
}

__device__ __forceinline__ void fixer_bar() { asm volatile("bar.sync 2, %0;" ::"n"(2 * 32) : "memory"); }

__device__ __forceinline__ bool ops_wait(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!umma::mbar_try_wait(bar, parity))
        if (clock64() - t0 > umma::kWaitCycles) {
            atomicExch(&g_ops_status, BLAZ_ERR_TIMEOUT);
            return false;
        }
    return true;
}

__device__ __forceinline__ void compute_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kAddTile) : "memory"); }

constexpr int kAddFixers = 2;  // fixer warps per CTA

template <bool kSub>
__global__ void __launch_bounds__(kAddTile + 32 * kAddFixers, kAddCtas)
    k_add_tile(int64_t nb, const double *f1, const double *s1, const uint8_t *p1, const int8_t *c1,
               const double *f2, const double *s2, const uint8_t *p2, const int8_t *c2, double *f, double *s,
               uint8_t *p, int8_t *c)
{
    // dynamic shared memory (kAddSmem bytes): input stages, output tiles, lists
    extern __shared__ __align__(16) uint8_t add_smem[];
    AddStage *stages = reinterpret_cast<AddStage *>(add_smem);
    uint32_t(*so_st)[kAddTile * 7] = reinterpret_cast<uint32_t(*)[kAddTile * 7]>(add_smem + kAddStages * sizeof(AddStage));
    AddFix(*fix)[kAddFixCap] = reinterpret_cast<AddFix(*)[kAddFixCap]>(
        add_smem + kAddStages * sizeof(AddStage) + kAddOut * kAddTile * 7 * 4);
    __shared__ int nfix[kAddOut];
    __shared__ __align__(8) uint64_t work_ready[kAddOut], out_free[kAddOut];
    __shared__ double fbeta[kAddFixers][kAddFixCap];  // beta_1, beta_2 of the listed blocks
    __shared__ volatile int fix_ok;
    __shared__ volatile int abort_flag;
    __shared__ volatile int go_on[2];  // written by thread 0 only, before the compute barrier
    const int t = threadIdx.x;
    const int64_t ntiles = (nb + kAddTile - 1) / kAddTile;
    if (t == 0) {
        for (int q = 0; q < kAddOut; ++q) {
            umma::mbar_init(&work_ready[q], kAddTile);
            umma::mbar_init(&out_free[q], 1);
            nfix[q] = 0;
        }
        abort_flag = 0;
        umma::mbar_init_fence();
    }
    __syncthreads();

    if (t >= kAddTile) {
        // the two fixer warps: fixer fw forms beta_(fw+1) of every listed
        // block, then the listed codes 4q+k with k of parity fw; both store
        // the tile
        const int fw = (t - kAddTile) >> 5, lane = t & 31, ft = t - kAddTile;
        for (int it = 0;; ++it) {
            const int64_t tile = blockIdx.x + (int64_t)it * gridDim.x;
            if (tile >= ntiles) break;
            const int u = it % kAddOut;
            // fixer 0 waits for the tile; both learn the outcome after one
            // barrier, so they always leave the loop together
            if (ft == 0) fix_ok = ops_wait(&work_ready[u], (it / kAddOut) & 1) ? 1 : 0;
            fixer_bar();
            if (!fix_ok) {
                abort_flag = 1;
                break;
            }
            const int n = min(nfix[u], kAddFixCap);
            for (int e = lane; e < n; e += 32) {
                const AddFix &x = fix[u][e];
                fbeta[fw][e] = add_fix_beta(fw ? x.sb : x.sa, x.ss, fw ? x.pb : x.pa, x.ph);
            }
            fixer_bar();
            for (int e = lane; e < n; e += 32) {
                const AddFix &x = fix[u][e];
                add_fix_codes<kSub>(fbeta[0][e], fbeta[1][e], x.wa, x.wb, x.undecided, fw, so_st[u] + x.t * 7);
            }
            fixer_bar();
            const int64_t b0 = tile * kAddTile;
            const int nt = (int)(nb - b0 < kAddTile ? nb - b0 : (int64_t)kAddTile);
            uint32_t *go = reinterpret_cast<uint32_t *>(c + b0 * kKeep);
            if (nt == kAddTile) {
                uint4 *vo = reinterpret_cast<uint4 *>(go);
                for (int i = ft; i < kAddTile * 7 / 4; i += 32 * kAddFixers)
                    __stcs(vo + i, reinterpret_cast<const uint4 *>(so_st[u])[i]);
            } else {
                for (int i = ft; i < nt * 7; i += 32 * kAddFixers) __stcs(go + i, so_st[u][i]);
            }
            fixer_bar();  // both warps' reads of the output tile and the list are done
            if (ft == 0) {
                nfix[u] = 0;
                umma::mbar_arrive(&out_free[u]);
            }
        }
        return;
    }

    // the compute warps: the inputs of kAddStages - 1 tiles in flight ahead
    // of the tile being decided
#pragma unroll
    for (int k = 0; k < kAddStages - 1; ++k) {
        const int64_t tk = blockIdx.x + (int64_t)k * gridDim.x;
        if (tk < ntiles) add_stage(tk, nb, f1, s1, p1, c1, f2, s2, p2, c2, stages[k], t);
        cp_async_commit();
    }
    int64_t tile = blockIdx.x;
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const int u = it % kAddOut;
        const AddStage &stg = stages[it % kAddStages];
        const uint32_t *sa_w = stg.ca, *sb_w = stg.cb;
        uint32_t *so_w = so_st[u];
        const int64_t b0 = tile * kAddTile;
        const int nt = (int)(nb - b0 < kAddTile ? nb - b0 : (int64_t)kAddTile);
        // output tile u is free once the fixers have stored tile it - kAddOut;
        // thread 0 takes the decision to go on for all compute threads (a
        // fixer may set abort_flag at any time: reading it after the barrier
        // could split the threads, and the next barrier has no time limit;
        // two copies, so that thread 0 never rewrites the one a thread may
        // still be about to read)
        if (t == 0) {
            if (!ops_wait(&out_free[u], ((it / kAddOut) & 1) ^ 1)) abort_flag = 1;
            go_on[it & 1] = !abort_flag;
        }
        cp_async_wait_stage();  // this thread's copies of the current stage have landed
        // the one barrier of the tile: every copy of this stage is visible,
        // and every thread is done with the stage of tile it - 1, which the
        // copies for tile it + kAddStages - 1 now refill
        compute_bar();
        if (!go_on[it & 1]) break;
        const int64_t ahead = tile + (int64_t)(kAddStages - 1) * gridDim.x;
        if (ahead < ntiles)
            add_stage(ahead, nb, f1, s1, p1, c1, f2, s2, p2, c2, stages[(it + kAddStages - 1) % kAddStages], t);
        cp_async_commit();
        if (t < nt) {
            const int64_t b = b0 + t;
            const double fa = stg.fa[t], fb = stg.fb[t], sa = stg.sa[t], sb = stg.sb[t];
            const int pa = stg.pa[t], pb = stg.pb[t];
            const double fs = kSub ? dsub(fa, fb) : dadd(fa, fb);
            const double ss = dadd(sa, sb);
            int ph = (pa * pb) / (pa + pb);
            ph = ph < 1 ? 1 : ph;
            uint32_t undecided = 0u;
            const unsigned hs = (unsigned)__double2hiint(ss), ls = (unsigned)__double2loint(ss);
            if (((hs & 0x7FFFFFFFu) | ls) == 0u) {  // s == 0: codes 0
#pragma unroll
                for (int q = 0; q < 7; ++q) so_w[t * 7 + q] = 0u;
            } else {
                const float phf = (float)ph;
                float b1f = 0.0f, b2f = 0.0f;
                const bool ok = beta_f32(sa, ss, __fdividef(phf, (float)pa), b1f) &
                                beta_f32(sb, ss, __fdividef(phf, (float)pb), b2f);
                const float E = __fmaf_rn(0x1.4p-12f, __fadd_rn(fabsf(b1f), fabsf(b2f)), 0x1p-100f);
                // two codes at a time on the paired fp32 pipe (same per-lane roundings)
                const float2 B1 = make_float2(b1f, b1f), B2 = make_float2(kSub ? -b2f : b2f, kSub ? -b2f : b2f);
                const float2 EP = make_float2(E, E), EN = make_float2(-E, -E);
                const float2 bias = make_float2(-12583040.0f, -12583040.0f);
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    // byte k of (w ^ 0x80808080) in the low byte of 1.5 2^23: the float 12583040 + c
                    const uint32_t wa = sa_w[t * 7 + q] ^ 0x80808080u, wb = sb_w[t * 7 + q] ^ 0x80808080u;
                    uint32_t lo8[4], hi8[4];
#pragma unroll
                    for (int k = 0; k < 4; k += 2) {
                        const float2 x1 = __fadd2_rn(make_float2(__uint_as_float(__byte_perm(wa, 0x4B400000u, 0x7640 + k)),
                                                                 __uint_as_float(__byte_perm(wa, 0x4B400000u, 0x7641 + k))),
                                                     bias);
                        const float2 x2 = __fadd2_rn(make_float2(__uint_as_float(__byte_perm(wb, 0x4B400000u, 0x7640 + k)),
                                                                 __uint_as_float(__byte_perm(wb, 0x4B400000u, 0x7641 + k))),
                                                     bias);
                        const float2 v = __ffma2_rn(B1, x1, __fmul2_rn(B2, x2));
                        const float2 hi = __fadd2_rn(v, EP), lo = __fadd2_rn(v, EN);
                        lo8[k] = cvt_s8_rz(lo.x);
                        lo8[k + 1] = cvt_s8_rz(lo.y);
                        hi8[k] = cvt_s8_rz(hi.x);
                        hi8[k + 1] = cvt_s8_rz(hi.y);
                    }
                    const uint32_t lw = __byte_perm(__byte_perm(lo8[0], lo8[1], 0x0040), __byte_perm(lo8[2], lo8[3], 0x0040), 0x5410);
                    const uint32_t hw = __byte_perm(__byte_perm(hi8[0], hi8[1], 0x0040), __byte_perm(hi8[2], hi8[3], 0x0040), 0x5410);
                    so_w[t * 7 + q] = lw;
                    undecided |= undecided_bytes(lw, hw) >> (7 - q);  // bit 8k + q
                }
                if (!ok) undecided = 0x7F7F7F7Fu;
            }
            if (undecided) {
                const int i = atomicAdd(&nfix[u], 1);
                if (i < kAddFixCap) {
                    AddFix &x = fix[u][i];
                    x.sa = sa;
                    x.sb = sb;
                    x.ss = ss;
#pragma unroll
                    for (int q = 0; q < 7; ++q) {
                        x.wa[q] = sa_w[t * 7 + q];
                        x.wb[q] = sb_w[t * 7 + q];
                    }
                    x.undecided = undecided;
                    x.t = t;
                    x.pa = pa;
                    x.pb = pb;
                    x.ph = ph;
                } else {
                    add_fix_block<kSub>(sa, sb, pa, pb, sa_w + t * 7, sb_w + t * 7, undecided, so_w + t * 7);
                }
            }
            __stcs(f + b, fs);
            __stcs(s + b, ss);
            p[b] = (uint8_t)ph;
        }
        umma::mbar_arrive(&work_ready[u]);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // nothing in flight at exit (an aborted loop)
}

// Algorithm 2.  When out == a (in place) only f and s are touched; otherwise
// phi and the codes are copied by the same kernel (one pass over the data).
template <bool kCopy>
__global__ void __launch_bounds__(256) k_scale(int64_t nb, const double *f1, const double *s1, const uint8_t *p1,
                                               const int8_t *c1, double cst, double *f, double *s, uint8_t *p,
                                               int8_t *c)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += stride) {
        f[b] = dmul(f1[b], cst);
        s[b] = dmul(s1[b], cst);
        if (kCopy) p[b] = p1[b];
    }
    if (kCopy) {
        // codes: nb*28 bytes = nb*7 32-bit words
        const uint32_t *src = reinterpret_cast<const uint32_t *>(c1);
        uint32_t *dst = reinterpret_cast<uint32_t *>(c);
        for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nb * 7; w += stride) dst[w] = src[w];
    }
}

// Algorithm 2 with 16-byte accesses (all four arrays of both matrices 16-byte
// aligned): f and s as pairs of binary64 products, phi and the codes copied
// as 16-byte words, the ragged tails of each array byte by byte.  Same bits
// as k_scale.
template <bool kCopy>
__global__ void __launch_bounds__(256)
    k_scale_vec(int64_t nb, const double *f1, const double *s1, const uint8_t *p1, const int8_t *c1, double cst,
                double *f, double *s, uint8_t *p, int8_t *c)  // f1 == f and s1 == s in place
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n2 = nb / 2;
    const double2 *f1v = reinterpret_cast<const double2 *>(f1), *s1v = reinterpret_cast<const double2 *>(s1);
    double2 *fv = reinterpret_cast<double2 *>(f), *sv = reinterpret_cast<double2 *>(s);
    for (int64_t i = tid; i < n2; i += stride) {
        double2 a = f1v[i], b = s1v[i];
        a.x = dmul(a.x, cst);
        a.y = dmul(a.y, cst);
        b.x = dmul(b.x, cst);
        b.y = dmul(b.y, cst);
        fv[i] = a;
        sv[i] = b;
    }
    if (tid == 0 && (nb & 1)) {
        f[nb - 1] = dmul(f1[nb - 1], cst);
        s[nb - 1] = dmul(s1[nb - 1], cst);
    }
    if (!kCopy) return;
    const int64_t np = nb / 16, nc = nb * kKeep / 16;
    const uint4 *p1v = reinterpret_cast<const uint4 *>(p1), *c1v = reinterpret_cast<const uint4 *>(c1);
    uint4 *pv = reinterpret_cast<uint4 *>(p), *cv = reinterpret_cast<uint4 *>(c);
    for (int64_t i = tid; i < np; i += stride) __stcs(pv + i, __ldcs(p1v + i));
    for (int64_t i = tid; i < nc; i += stride) __stcs(cv + i, __ldcs(c1v + i));
    for (int64_t i = np * 16 + tid; i < nb; i += stride) p[i] = p1[i];
    for (int64_t i = nc * 16 + tid; i < nb * kKeep; i += stride) c[i] = c1[i];
}

static int grid_for(int64_t n, int threads)
{
    int64_t want = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 32;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

int ops_device_status()
{
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_ops_status, sizeof(int));
    if (e != cudaSuccess) return set_cuda_error(e);
    if (v != 0) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_ops_status, &zero, sizeof(int));
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return v;
}

int launch_add(const blaz_cmat *a, const blaz_cmat *b, const blaz_cmat *o, bool subtract, cudaStream_t st)
{
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    if (nb == 0) return BLAZ_OK;
    auto a16 = [](const void *q) { return ((uintptr_t)q & 15) == 0; };
    if (a16(a->code) && a16(b->code) && a16(o->code) && a16(a->f) && a16(b->f) && a16(a->s) && a16(b->s) &&
        a16(a->phi) && a16(b->phi)) {
        // one wave of kAddCtas resident CTAs per SM, each looping over its
        // tiles with the inputs of the next kAddStages - 1 tiles in flight
        const int64_t ntiles = (nb + kAddTile - 1) / kAddTile;
        const int grid = (int)std::min<int64_t>(ntiles, (int64_t)num_sms() * kAddCtas);
        static const bool smem_ok = [] {
            return cudaFuncSetAttribute(k_add_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kAddSmem) == cudaSuccess &&
                   cudaFuncSetAttribute(k_add_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kAddSmem) == cudaSuccess;
        }();
        if (!smem_ok) return set_cuda_error(cudaGetLastError());
        if (subtract)
            k_add_tile<true><<<grid, kAddTile + 32 * kAddFixers, kAddSmem, st>>>(nb, a->f, a->s, a->phi, a->code, b->f, b->s, b->phi,
                                                        b->code, o->f, o->s, o->phi, o->code);
        else
            k_add_tile<false><<<grid, kAddTile + 32 * kAddFixers, kAddSmem, st>>>(nb, a->f, a->s, a->phi, a->code, b->f, b->s, b->phi,
                                                         b->code, o->f, o->s, o->phi, o->code);
        return launch_status();
    }
    const int grid = grid_for(nb, 128);
    if (subtract)
        k_add<true><<<grid, 128, 0, st>>>(nb, a->f, a->s, a->phi, a->code, b->f, b->s, b->phi, b->code, o->f, o->s,
                                          o->phi, o->code);
    else
        k_add<false><<<grid, 128, 0, st>>>(nb, a->f, a->s, a->phi, a->code, b->f, b->s, b->phi, b->code, o->f, o->s,
                                           o->phi, o->code);
    return launch_status();
}

int launch_scale(const blaz_cmat *a, double c, const blaz_cmat *o, cudaStream_t st)
{
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    if (nb == 0) return BLAZ_OK;
    const bool copy = o->code != a->code || o->phi != a->phi;
    auto a16 = [](const void *q) { return ((uintptr_t)q & 15) == 0; };
    const bool vec = a16(a->f) && a16(a->s) && a16(o->f) && a16(o->s) &&
                     (!copy || (a16(a->phi) && a16(a->code) && a16(o->phi) && a16(o->code)));
    if (vec) {
        // one 16-byte word per thread and pass: 4 resident CTAs of 256 threads per SM, two waves
        const int grid = (int)std::min<int64_t>((int64_t)num_sms() * 8, std::max<int64_t>(1, (nb * 7 / 4 + 255) / 256));
        if (copy)
            k_scale_vec<true><<<grid, 256, 0, st>>>(nb, a->f, a->s, a->phi, a->code, c, o->f, o->s, o->phi, o->code);
        else
            k_scale_vec<false><<<grid, 256, 0, st>>>(nb, a->f, a->s, a->phi, a->code, c, o->f, o->s, o->phi, o->code);
    } else if (copy) {
        k_scale<true><<<grid_for(nb * 7, 256), 256, 0, st>>>(nb, a->f, a->s, a->phi, a->code, c, o->f, o->s, o->phi,
                                                           o->code);
    } else {
        k_scale<false><<<grid_for(nb, 256), 256, 0, st>>>(nb, a->f, a->s, a->phi, a->code, c, o->f, o->s, o->phi,
                                                            o->code);
    }
    return launch_status();
}

}  // namespace blaz
