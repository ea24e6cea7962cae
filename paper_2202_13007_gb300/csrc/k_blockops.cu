// k_blockops.cu -- operations on compressed blocks without decompression:
// addition / subtraction (Algorithm 1, Eq. eq55) and multiplication by a
// constant (Algorithm 2) of "Compressed Matrix Computations" (arXiv 2202.13007).
// Bit-exact binary64 (explicit round-to-nearest intrinsics).
#include <algorithm>

#include "block_ops.cuh"

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

// fp32 estimate of beta_k = RN(RN(RN(s_k / s) / phi_k) * phi) (Algorithm 1)
// for the tiled addition below; rho = phi / phi_k, evaluated in fp32.
//   s_k and s are truncated to fp32 after scaling both by 2^-e(s) (exponent
//   arithmetic on the integer pipe, exact): relative error < 2^-23 each;
//   __fdividef: < 2^-22; rho: < 2^-22; the product: < 2^-24.  So
//   |beta - beta_k| < (2^-21 + 2^-22 + 2^-24)(1 + 2^-20) |beta_k| < 2^-20 |beta_k|
//   (the three binary64 roundings of beta_k are below 2^-51 relative).
// s_k == 0 gives beta = 0 exactly (beta_k is a signed zero).  Returns false
// when s_k or s is subnormal, Inf or NaN, or when |s_k / s| leaves
// [2^-100, 2^101): the caller then evaluates beta_k in binary64.
__device__ __forceinline__ bool beta_f32(double sk, double ss, float rho, float &beta)
{
    const unsigned hk = (unsigned)__double2hiint(sk), lk = (unsigned)__double2loint(sk);
    const unsigned hs = (unsigned)__double2hiint(ss), ls = (unsigned)__double2loint(ss);
    if (((hk & 0x7FFFFFFFu) | lk) == 0u) {
        beta = 0.0f;
        return true;
    }
    const int ek = (int)((hk >> 20) & 0x7FF), es = (int)((hs >> 20) & 0x7FF);
    const int d = ek - es;
    if (ek == 0 || ek == 0x7FF || es == 0 || es == 0x7FF || d < -100 || d > 100) return false;
    const float xk = __uint_as_float((hk & 0x80000000u) | ((unsigned)(d + 127) << 23) |
                                     (__funnelshift_l(lk, hk, 3) & 0x7FFFFFu));
    const float xs = __uint_as_float((hs & 0x80000000u) | (127u << 23) | (__funnelshift_l(ls, hs, 3) & 0x7FFFFFu));
    beta = __fmul_rn(__fdividef(xk, xs), rho);
    return true;
}

// Algorithm 1 over tiles of kAddTile blocks with the four binary64 divisions
// taken out of the common path.  Each CTA stages the codes of both operands
// with coalesced 16-byte loads into shared memory (a thread's 28 codes are
// then 7 words at stride 7: conflict-free), forms beta_k in fp32 (beta_f32)
// and decides each code from v = fl(beta_1 c_1 +- beta_2 c_2) and the bound
//   |v - y| <= 2^-19 (|beta_1 c_1| + |beta_2 c_2|) + 2^-22 |v| + 2^-100
// (2^-20 from beta, 2^-23 from the fp32 product and fma, the binary64
// roundings of the specification far below), as add_block_fast does with
// its tighter bound.  f and s are two binary64 additions per block.
//
// A block with an undecided code, or whose beta_k has no fp32 estimate, is
// appended to a per-tile list; after a barrier the CTA's threads evaluate
// the listed blocks densely, one per thread, in binary64 (add_block's
// arithmetic) for the undecided codes only.  Undecided codes are structural
// rather than rare: equal phi and equal codes in both operands put y on an
// integer (y = c phi / phi_k in real arithmetic), about one block in ten of
// two smooth fields, so the dense list keeps the binary64 divisions to the
// blocks that need them instead of to every warp that holds one.
//
// Output codes leave through shared memory as 16-byte stores.  Every input
// of a tile is read before any output of it is written, so out may alias a
// or b.  Requires 16-byte aligned code arrays (the launcher checks).
constexpr int kAddTile = 256;

struct AddFix {
    double sa, sb;
    uint32_t undecided;  // bit 4q+k: code 4q+k
    int t, pa, pb;
};

template <bool kSub>
__global__ void __launch_bounds__(kAddTile, 4)
    k_add_tile(int64_t nb, const double *f1, const double *s1, const uint8_t *p1, const int8_t *c1,
               const double *f2, const double *s2, const uint8_t *p2, const int8_t *c2, double *f, double *s,
               uint8_t *p, int8_t *c)
{
    __shared__ __align__(16) uint32_t sa_w[kAddTile * 7];
    __shared__ __align__(16) uint32_t sb_w[kAddTile * 7];
    __shared__ __align__(16) uint32_t so_w[kAddTile * 7];
    __shared__ AddFix fix[kAddTile];
    __shared__ int nfix;
    const int t = threadIdx.x;
    const int64_t ntiles = (nb + kAddTile - 1) / kAddTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t b0 = tile * kAddTile;
        const int nt = (int)(nb - b0 < kAddTile ? nb - b0 : (int64_t)kAddTile);
        const int nw = nt * 7;  // 32-bit words of codes in this tile
        const uint32_t *ga = reinterpret_cast<const uint32_t *>(c1 + b0 * kKeep);
        const uint32_t *gb = reinterpret_cast<const uint32_t *>(c2 + b0 * kKeep);
        if (t == 0) nfix = 0;
        if (nt == kAddTile) {
            const uint4 *va = reinterpret_cast<const uint4 *>(ga), *vb = reinterpret_cast<const uint4 *>(gb);
            for (int i = t; i < kAddTile * 7 / 4; i += kAddTile) {
                reinterpret_cast<uint4 *>(sa_w)[i] = __ldcs(va + i);
                reinterpret_cast<uint4 *>(sb_w)[i] = __ldcs(vb + i);
            }
        } else {
            for (int i = t; i < nw; i += kAddTile) {
                sa_w[i] = __ldcs(ga + i);
                sb_w[i] = __ldcs(gb + i);
            }
        }
        const int64_t b = b0 + t;
        double fa = 0.0, fb = 0.0, sa = 0.0, sb = 0.0;
        int pa = 1, pb = 1;
        if (t < nt) {
            fa = __ldcs(f1 + b);
            fb = __ldcs(f2 + b);
            sa = __ldcs(s1 + b);
            sb = __ldcs(s2 + b);
            pa = __ldcs(p1 + b);
            pb = __ldcs(p2 + b);
        }
        __syncthreads();
        if (t < nt) {
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
                const float ab1 = fabsf(b1f), ab2 = fabsf(b2f);
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    const uint32_t wa = sa_w[t * 7 + q], wb = sb_w[t * 7 + q];
                    uint32_t v32 = 0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int i1 = (int)(int8_t)(uint8_t)(wa >> (8 * k));
                        const int i2 = (int)(int8_t)(uint8_t)(wb >> (8 * k));
                        const float x1 = small_int_to_float(i1), x2 = small_int_to_float(i2);
                        const float v = fmaf(b1f, x1, kSub ? -(b2f * x2) : b2f * x2);
                        const float E = 0x1p-19f * fmaf(ab1, fabsf(x1), ab2 * fabsf(x2)) + 0x1p-22f * fabsf(v) +
                                        0x1p-100f;
                        const float lo = v - E, hi = v + E;
                        int code;
                        bool done;
                        if (lo >= 127.0f) {
                            code = 127;
                            done = true;
                        } else if (hi <= -127.0f) {
                            code = -127;
                            done = true;
                        } else {
                            const int tl = (int)truncf(lo), th = (int)truncf(hi);
                            code = tl;
                            done = tl == th;
                        }
                        if (!done) undecided |= 1u << (4 * q + k);
                        v32 |= (uint32_t)(uint8_t)(int8_t)code << (8 * k);
                    }
                    so_w[t * 7 + q] = v32;
                }
                if (!ok) undecided = 0x0FFFFFFFu;
            }
            if (undecided) {
                const int i = atomicAdd(&nfix, 1);
                fix[i].sa = sa;
                fix[i].sb = sb;
                fix[i].undecided = undecided;
                fix[i].t = t;
                fix[i].pa = pa;
                fix[i].pb = pb;
            }
            __stcs(f + b, fs);
            __stcs(s + b, ss);
            p[b] = (uint8_t)ph;
        }
        __syncthreads();
        // binary64 Algorithm 1 for the undecided codes of the listed blocks
        for (int i = t; i < nfix; i += kAddTile) {
            const AddFix e = fix[i];
            const double ss = dadd(e.sa, e.sb);
            int ph = (e.pa * e.pb) / (e.pa + e.pb);
            ph = ph < 1 ? 1 : ph;
            const double a1 = ddiv(e.sa, ss);
            const double a2 = ddiv(e.sb, ss);
            const double phd = i64_to_double(ph);
            const double b1 = dmul(div_small_int(a1, e.pa), phd);
            const double b2 = dmul(div_small_int(a2, e.pb), phd);
            for (int q = 0; q < 7; ++q) {
                const uint32_t m = (e.undecided >> (4 * q)) & 0xFu;
                if (!m) continue;
                const uint32_t wa = sa_w[e.t * 7 + q], wb = sb_w[e.t * 7 + q];
                uint32_t w = so_w[e.t * 7 + q];
                for (int k = 0; k < 4; ++k)
                    if (m & (1u << k)) {
                        const double x1 = (double)(int8_t)(uint8_t)(wa >> (8 * k));
                        const double x2 = (double)(int8_t)(uint8_t)(wb >> (8 * k));
                        const double y = kSub ? dsub(dmul(b1, x1), dmul(b2, x2)) : dadd(dmul(b1, x1), dmul(b2, x2));
                        w = (w & ~(0xFFu << (8 * k))) | ((uint32_t)(uint8_t)quantize(y) << (8 * k));
                    }
                so_w[e.t * 7 + q] = w;
            }
        }
        __syncthreads();
        uint32_t *go = reinterpret_cast<uint32_t *>(c + b0 * kKeep);
        if (nt == kAddTile) {
            uint4 *vo = reinterpret_cast<uint4 *>(go);
            for (int i = t; i < kAddTile * 7 / 4; i += kAddTile) __stcs(vo + i, reinterpret_cast<const uint4 *>(so_w)[i]);
        } else {
            for (int i = t; i < nw; i += kAddTile) __stcs(go + i, so_w[i]);
        }
        __syncthreads();
    }
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

int launch_add(const blaz_cmat *a, const blaz_cmat *b, const blaz_cmat *o, bool subtract, cudaStream_t st)
{
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    if (nb == 0) return BLAZ_OK;
    auto a16 = [](const void *q) { return ((uintptr_t)q & 15) == 0; };
    if (a16(a->code) && a16(b->code) && a16(o->code)) {
        // tiles of 256 blocks; 4 resident CTAs per SM, a few waves of tiles
        const int64_t ntiles = (nb + kAddTile - 1) / kAddTile;
        const int grid = (int)std::min<int64_t>(ntiles, (int64_t)num_sms() * 4 * 4);
        if (subtract)
            k_add_tile<true><<<grid, kAddTile, 0, st>>>(nb, a->f, a->s, a->phi, a->code, b->f, b->s, b->phi,
                                                        b->code, o->f, o->s, o->phi, o->code);
        else
            k_add_tile<false><<<grid, kAddTile, 0, st>>>(nb, a->f, a->s, a->phi, a->code, b->f, b->s, b->phi,
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
