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
// The kernels are the plain binary64 forms, one thread per block, in the
// binary64 operation order of the 28-code compressor (bit-identical codes);
// the rate-2 format keeps its certified fast kernels.
#include "block_codec.cuh"

namespace blaz {

__host__ __device__ constexpr int rate_keep(int r) { return 8 * r + (8 - r) * r; }

// Kept index of coefficient (i, j) at rate r, or -1.
__device__ __forceinline__ int rate_index(int r, int i, int j)
{
    return i < r ? i * 8 + j : (j < r ? 8 * r + (i - r) * r + j : -1);
}

// The DCT column j of D' (Eq. eqdct, one column at a time as compress_block
// forms it): X[i] = RN(aa_ij U_ij), U_ij = sum_u cos_iu T_u, T_u = sum_v
// D'_uv cos_jv (products by cos(0) = 1 are exact and omitted).
__device__ __forceinline__ void dct_column(const double (&d)[64], int j, double (&X)[8])
{
    double T[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        double acc = (j == 0) ? d[u * 8] : dmul(d[u * 8], cos_tab(j, 0));
#pragma unroll
        for (int v = 1; v < 8; ++v) acc = dadd(acc, (j == 0) ? d[u * 8 + v] : dmul(d[u * 8 + v], cos_tab(j, v)));
        T[u] = acc;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        double acc = (i == 0) ? T[0] : dmul(cos_tab(i, 0), T[0]);
#pragma unroll
        for (int u = 1; u < 8; ++u) acc = dadd(acc, (i == 0) ? T[u] : dmul(cos_tab(i, u), T[u]));
        X[i] = dmul(aa_tab(i, j), acc);
    }
}

__global__ void __launch_bounds__(128)
    k_compress_rate(const double *__restrict__ A, int64_t lda, int64_t nbc, int64_t nb, int r, double *f, double *s,
                    uint8_t *phi, int8_t *code)
{
    const int nk = rate_keep(r);
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bi = b / nbc, bj = b - bi * nbc;
        double d[64];
        load_block<false>(A, lda, bi, bj, d);
        f[b] = d[0];
        // Eq. eqnorm, in place from the last element backwards
#pragma unroll
        for (int i = 7; i >= 0; --i)
#pragma unroll
            for (int j = 7; j >= 0; --j) {
                if (i == 0 && j == 0) d[0] = 0.0;
                else if (i == 0) d[j] = dsub(d[j], d[j - 1]);
                else if (j == 0) d[i * 8] = dsub(d[i * 8], d[(i - 1) * 8]);
                else d[i * 8 + j] = dmul(dadd(dsub(d[i * 8 + j], d[(i - 1) * 8 + j]), dsub(d[i * 8 + j], d[i * 8 + j - 1])), 0.5);
            }
        int K = 0;
#pragma unroll
        for (int p = 0; p < 64; ++p) K += (d[p] != 0.0);
        const double S = tree_sum_abs(d);
        int8_t *cb = code + b * nk;
        if (K == 0) {  // constant block: s = 0, codes 0, phi = 255
            s[b] = 0.0;
            phi[b] = 255;
            for (int t = 0; t < nk; ++t) cb[t] = 0;
            continue;
        }
        const double sv = ddiv(S, (double)K);
        const double rv = ddiv(1.0, sv);
#pragma unroll
        for (int p = 0; p < 64; ++p) d[p] = dmul(d[p], rv);
        s[b] = sv;
        // Eq. eqphi from all 64 coefficients, then the kept codes (the
        // columns are evaluated again: a second pass instead of 64 more
        // registers)
        double m = 0.0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            double X[8];
            dct_column(d, j, X);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const double ax = fabs(X[i]);
                m = (ax > m) ? ax : m;
            }
        }
        const double q = ddiv(127.0, m);
        int ph;
        if (!(q < 255.0)) ph = 255;
        else {
            ph = __double2int_rz(q);
            ph = ph < 1 ? 1 : ph;
        }
        phi[b] = (uint8_t)ph;
        const double phd = (double)ph;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            double X[8];
            dct_column(d, j, X);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int t = rate_index(r, i, j);
                if (t >= 0) cb[t] = quantize(dmul(X[i], phd));
            }
        }
    }
}

// Decompression of a rate-r block: X = code / phi on the kept positions, the
// inverse DCT (Y = aa X; Q = Y cos; P = cos^T Q), times s, then the exact
// inverse of Eq. eqnorm.  Within 1e-12 of the block's scale of the binary64
// evaluation of the definition.
__global__ void __launch_bounds__(128)
    k_decompress_rate(const double *__restrict__ f, const double *__restrict__ s, const uint8_t *__restrict__ phi,
                      const int8_t *__restrict__ code, int64_t nbc, int64_t nb, int r, double *A, int64_t lda)
{
    const int nk = rate_keep(r);
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bi = b / nbc, bj = b - bi * nbc;
        const int8_t *cb = code + b * nk;
        const double inv = 1.0 / (double)phi[b];
        double Y[64];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int t = rate_index(r, i, j);
                Y[i * 8 + j] = t >= 0 ? aa_tab(i, j) * ((double)cb[t] * inv) : 0.0;
            }
        double P[64];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            double Q[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                double acc = Y[i * 8] * cos_tab(0, v);
#pragma unroll
                for (int j = 1; j < 8; ++j) acc = fma(Y[i * 8 + j], cos_tab(j, v), acc);
                Q[i] = acc;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                double acc = cos_tab(0, u) * Q[0];
#pragma unroll
                for (int i = 1; i < 8; ++i) acc = fma(cos_tab(i, u), Q[i], acc);
                P[u * 8 + v] = acc;
            }
        }
        const double sv = s[b];
        double M[64];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const double dh = sv * P[i * 8 + j];
                double v;
                if (i == 0 && j == 0) v = f[b];
                else if (i == 0) v = M[j - 1] + dh;
                else if (j == 0) v = M[(i - 1) * 8] + dh;
                else v = (M[(i - 1) * 8 + j] + M[i * 8 + j - 1]) * 0.5 + dh;
                M[i * 8 + j] = v;
            }
        double *p = A + (bi * 8) * lda + bj * 8;
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) p[i * lda + j] = M[i * 8 + j];
    }
}

// Algorithm 1 (kSub: the subtraction) on rate-r blocks, in the binary64
// order of add_block; every input of a block is read before its outputs are
// written, so out may alias a or b.
template <bool kSub>
__global__ void __launch_bounds__(128)
    k_add_rate(int64_t nb, int r, const double *f1, const double *s1, const uint8_t *p1, const int8_t *c1,
               const double *f2, const double *s2, const uint8_t *p2, const int8_t *c2, double *f, double *s,
               uint8_t *p, int8_t *c)
{
    const int nk = rate_keep(r);
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const double fa = f1[b], fb = f2[b], sa = s1[b], sb = s2[b];
        const int pa = p1[b], pb = p2[b];
        const double fs = kSub ? dsub(fa, fb) : dadd(fa, fb);
        const double ss = dadd(sa, sb);
        int ph = (pa * pb) / (pa + pb);
        ph = ph < 1 ? 1 : ph;
        const int8_t *ca = c1 + b * nk, *cbb = c2 + b * nk;
        int8_t *co = c + b * nk;
        if (ss == 0.0) {
            for (int t = 0; t < nk; ++t) co[t] = 0;
        } else {
            const double a1 = ddiv(sa, ss), a2 = ddiv(sb, ss);
            const double phd = (double)ph;
            const double b1 = dmul(ddiv(a1, (double)pa), phd), b2 = dmul(ddiv(a2, (double)pb), phd);
            for (int t = 0; t < nk; ++t) {
                const double x1 = (double)ca[t], x2 = (double)cbb[t];
                co[t] = quantize(kSub ? dsub(dmul(b1, x1), dmul(b2, x2)) : dadd(dmul(b1, x1), dmul(b2, x2)));
            }
        }
        f[b] = fs;
        s[b] = ss;
        p[b] = (uint8_t)ph;
    }
}

// Algorithm 2 on rate-r blocks: f and s times c; phi and the codes copied
// (untouched when out is a).
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
    if (copy)
        for (int64_t i = tid; i < nb * rate_keep(r); i += stride) c[i] = c1[i];
}

static int rate_grid(int64_t n, int threads)
{
    const int64_t want = (n + threads - 1) / threads, cap = (int64_t)num_sms() * 16;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

int launch_compress_rate(const double *A, int64_t lda, const blaz_cmat *out, int r, cudaStream_t st)
{
    const int64_t nbc = out->cols / 8, nb = (out->rows / 8) * nbc;
    if (nb == 0) return BLAZ_OK;
    k_compress_rate<<<rate_grid(nb, 128), 128, 0, st>>>(A, lda, nbc, nb, r, out->f, out->s, out->phi, out->code);
    return launch_status();
}

int launch_decompress_rate(const blaz_cmat *a, int r, double *A, int64_t lda, cudaStream_t st)
{
    const int64_t nbc = a->cols / 8, nb = (a->rows / 8) * nbc;
    if (nb == 0) return BLAZ_OK;
    k_decompress_rate<<<rate_grid(nb, 128), 128, 0, st>>>(a->f, a->s, a->phi, a->code, nbc, nb, r, A, lda);
    return launch_status();
}

int launch_add_rate(const blaz_cmat *a, const blaz_cmat *b, const blaz_cmat *o, int r, bool subtract,
                    cudaStream_t st)
{
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    if (nb == 0) return BLAZ_OK;
    if (subtract)
        k_add_rate<true><<<rate_grid(nb, 128), 128, 0, st>>>(nb, r, a->f, a->s, a->phi, a->code, b->f, b->s,
                                                             b->phi, b->code, o->f, o->s, o->phi, o->code);
    else
        k_add_rate<false><<<rate_grid(nb, 128), 128, 0, st>>>(nb, r, a->f, a->s, a->phi, a->code, b->f, b->s,
                                                              b->phi, b->code, o->f, o->s, o->phi, o->code);
    return launch_status();
}

int launch_scale_rate(const blaz_cmat *a, double cst, const blaz_cmat *o, int r, cudaStream_t st)
{
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    if (nb == 0) return BLAZ_OK;
    const bool copy = o->code != a->code || o->phi != a->phi;
    k_scale_rate<<<rate_grid(nb * rate_keep(r), 256), 256, 0, st>>>(nb, r, a->f, a->s, a->phi, a->code, cst, o->f,
                                                                    o->s, o->phi, o->code, copy);
    return launch_status();
}

}  // namespace blaz
