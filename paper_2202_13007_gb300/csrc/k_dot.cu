// k_dot.cu -- dot products on compressed matrices ("Dot product", Sec. III of
// "Compressed Matrix Computations", arXiv 2202.13007):
//   * the flattened product <vec A_hat, vec B_hat> of two same-shape matrices;
//   * Algorithm 3 (Eqs. eqbbb0, eqbbb): line i of A_hat times column j of B_hat.
// Both partly decompress the blocks they touch.  Reductions follow a fixed
// tree, so results are bitwise reproducible run to run.
#include "block_codec.cuh"

namespace blaz {

constexpr int kDotThreads = 256;

// Fixed-order CTA sum (warp shuffle tree, then the per-warp sums in order).
__device__ __forceinline__ double cta_sum(double v, double *red)
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

// Flattened dot.  Every CTA writes its partial sum; the last CTA to finish
// adds the partials in CTA order and resets the arrival counter.
__global__ void __launch_bounds__(kDotThreads)
    k_dot(int64_t nb, const double *__restrict__ fa, const double *__restrict__ sa, const uint8_t *__restrict__ pa,
          const int8_t *__restrict__ ca, const double *__restrict__ fb, const double *__restrict__ sb,
          const uint8_t *__restrict__ pb, const int8_t *__restrict__ cb, double *__restrict__ partials,
          unsigned *__restrict__ counter, double *__restrict__ result)
{
    __shared__ double red[kDotThreads / 32];
    __shared__ bool last;
    double acc = 0.0;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        double x[64], y[64];
        decompress_block_at(fa[b], sa[b], pa[b], ca + b * kKeep, x);
        decompress_block_at(fb[b], sb[b], pb[b], cb + b * kKeep, y);
        double blk = 0.0;
#pragma unroll
        for (int p = 0; p < 64; ++p) blk = fma(x[p], y[p], blk);
        acc += blk;
    }
    const double tot = cta_sum(acc, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = tot;
        __threadfence();
        const unsigned arrived = atomicAdd(counter, 1u);
        last = (arrived == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) v += __ldcg(partials + q);
    const double r = cta_sum(v, red);
    if (threadIdx.x == 0) {
        *result = r;
        *counter = 0u;
    }
}

// Algorithm 3 generalised to matrices: one CTA; thread t handles k-blocks
// t, t + blockDim, ...; each decompresses block (bi, kb) of A and (kb, bj) of B.
__global__ void __launch_bounds__(kDotThreads)
    k_dot_rowcol(int64_t nkb, int64_t nbc_a, int64_t nbc_b, int64_t i, int64_t j, const double *__restrict__ fa,
                 const double *__restrict__ sa, const uint8_t *__restrict__ pa, const int8_t *__restrict__ ca,
                 const double *__restrict__ fb, const double *__restrict__ sb, const uint8_t *__restrict__ pb,
                 const int8_t *__restrict__ cb, double *__restrict__ result)
{
    __shared__ double red[kDotThreads / 32];
    const int64_t bi = i / 8, bj = j / 8;
    const int ri = (int)(i % 8), cj = (int)(j % 8);
    double acc = 0.0;
    for (int64_t kb = threadIdx.x; kb < nkb; kb += blockDim.x) {
        const int64_t ba = bi * nbc_a + kb, bb = kb * nbc_b + bj;
        double x[64], y[64];
        decompress_block_at(fa[ba], sa[ba], pa[ba], ca + ba * kKeep, x);
        decompress_block_at(fb[bb], sb[bb], pb[bb], cb + bb * kKeep, y);
        double blk = 0.0;
#pragma unroll
        for (int t = 0; t < 8; ++t) blk = fma(x[ri * 8 + t], y[t * 8 + cj], blk);
        acc += blk;
    }
    const double r = cta_sum(acc, red);
    if (threadIdx.x == 0) *result = r;
}

int dot_grid(int64_t nb)
{
    int64_t want = (nb + kDotThreads - 1) / kDotThreads;
    int64_t cap = (int64_t)num_sms() * 4;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

int launch_dot(const blaz_cmat *a, const blaz_cmat *b, double *result, double *partials, unsigned *counter,
               int64_t max_ctas, cudaStream_t st)
{
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    int grid = dot_grid(nb);
    if (grid > max_ctas) grid = (int)max_ctas;
    k_dot<<<grid, kDotThreads, 0, st>>>(nb, a->f, a->s, a->phi, a->code, b->f, b->s, b->phi, b->code, partials,
                                        counter, result);
    return launch_status();
}

int launch_dot_rowcol(const blaz_cmat *a, const blaz_cmat *b, int64_t i, int64_t j, double *result, cudaStream_t st)
{
    k_dot_rowcol<<<1, kDotThreads, 0, st>>>(a->cols / 8, a->cols / 8, b->cols / 8, i, j, a->f, a->s, a->phi, a->code,
                                            b->f, b->s, b->phi, b->code, result);
    return launch_status();
}

}  // namespace blaz
