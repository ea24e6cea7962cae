// k_blockops.cu -- operations on compressed blocks without decompression:
// addition / subtraction (Algorithm 1, Eq. eq55) and multiplication by a
// constant (Algorithm 2) of "Compressed Matrix Computations" (arXiv 2202.13007).
// Bit-exact binary64 (explicit round-to-nearest intrinsics).
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
    if (o->code != a->code || o->phi != a->phi)
        k_scale<true><<<grid_for(nb * 7, 256), 256, 0, st>>>(nb, a->f, a->s, a->phi, a->code, c, o->f, o->s, o->phi,
                                                           o->code);
    else
        k_scale<false><<<grid_for(nb, 256), 256, 0, st>>>(nb, a->f, a->s, a->phi, a->code, c, o->f, o->s, o->phi,
                                                            o->code);
    return launch_status();
}

}  // namespace blaz
