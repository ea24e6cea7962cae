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
