// k_codec.cu -- compressor and decompressor kernels (Sec. II of "Compressed
// Matrix Computations", arXiv 2202.13007).
//
// Compression is bit-exact binary64: every operation is an explicit
// round-to-nearest intrinsic in the order fixed in include/blaz.h, so the
// result does not depend on -fmad or on the compiler's scheduling.
#include "block_codec.cuh"

namespace blaz {

// One thread per 8x8 block.  Loads the block (eight rows of 64 B) with 16-byte
// vector loads when the matrix allows it.
template <bool kVec>
__device__ __forceinline__ void load_block(const double *__restrict__ A, int64_t lda, int64_t bi, int64_t bj,
                                           double (&d)[64])
{
    const double *p = A + (bi * 8) * lda + bj * 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (kVec) {
            const double2 *q = reinterpret_cast<const double2 *>(p + i * lda);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                double2 v = __ldg(q + h);
                d[i * 8 + 2 * h] = v.x;
                d[i * 8 + 2 * h + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) d[i * 8 + j] = __ldg(p + i * lda + j);
        }
    }
}

// Compress one block held in d (overwritten).  Writes s, phi and the 28 codes.
__device__ __forceinline__ void compress_block(double (&d)[64], double &s_out, uint8_t &phi_out,
                                               int8_t (&code)[kKeep])
{
    // Eq. eqnorm, evaluated in place from the last element backwards so that
    // M(i-1,j) and M(i,j-1) are still the inputs when D(i,j) is formed.
#pragma unroll
    for (int i = 7; i >= 0; --i) {
#pragma unroll
        for (int j = 7; j >= 0; --j) {
            if (i == 0 && j == 0) {
                d[0] = 0.0;
            } else if (i == 0) {
                d[j] = dsub(d[j], d[j - 1]);
            } else if (j == 0) {
                d[i * 8] = dsub(d[i * 8], d[(i - 1) * 8]);
            } else {
                double a = dsub(d[i * 8 + j], d[(i - 1) * 8 + j]);
                double b = dsub(d[i * 8 + j], d[i * 8 + j - 1]);
                d[i * 8 + j] = dmul(dadd(a, b), 0.5);
            }
        }
    }
    // Eqs. eqslope / eqslope2: K nonzero entries, S = sum |D| row-major.
    int K = 0;
    double S = 0.0;
#pragma unroll
    for (int p = 0; p < 64; ++p) {
        K += (d[p] != 0.0);
        S = dadd(S, fabs(d[p]));
    }
    if (K == 0) {  // constant block: s = 0, all coefficients 0, phi = 127/0 -> 255
        s_out = 0.0;
        phi_out = 255;
#pragma unroll
        for (int t = 0; t < kKeep; ++t) code[t] = 0;
        return;
    }
    const double s = ddiv(S, (double)K);
    const double r = ddiv(1.0, s);
#pragma unroll
    for (int p = 0; p < 64; ++p) d[p] = dmul(d[p], r);
    s_out = s;

    // Eq. eqdct, one output column j at a time: inner sums T[u] over v, outer
    // sums over u, then the alpha_i alpha_j factor.  Multiplications by
    // cos(0) = 1 are exact and therefore omitted.
    double kept[kKeep];
    double m = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
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
            const double X = dmul(aa_tab(i, j), acc);
            const double ax = fabs(X);
            m = (ax > m) ? ax : m;
            const int t = kept_index(i, j);
            if (t >= 0) kept[t] = X;
        }
    }
    // Eq. eqphi
    const double q = ddiv(127.0, m);
    int phi;
    if (!(q < 255.0)) phi = 255;
    else {
        phi = __double2int_rz(q);
        phi = phi < 1 ? 1 : phi;
    }
    phi_out = (uint8_t)phi;
    const double phid = (double)phi;
#pragma unroll
    for (int t = 0; t < kKeep; ++t) code[t] = quantize(dmul(kept[t], phid));
}

template <bool kVec>
__global__ void __launch_bounds__(128) k_compress(const double *__restrict__ A, int64_t lda, int64_t nbc, int64_t nb,
                                                  double *__restrict__ f, double *__restrict__ s,
                                                  uint8_t *__restrict__ phi, int8_t *__restrict__ code)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bi = b / nbc, bj = b - (b / nbc) * nbc;
        double d[64];
        load_block<kVec>(A, lda, bi, bj, d);
        f[b] = d[0];
        double sv;
        uint8_t ph;
        int8_t c[kKeep];
        compress_block(d, sv, ph, c);
        s[b] = sv;
        phi[b] = ph;
        store_codes(code + b * kKeep, c);
    }
}

template <bool kVec>
__global__ void __launch_bounds__(128) k_decompress(const double *__restrict__ f, const double *__restrict__ s,
                                                    const uint8_t *__restrict__ phi,
                                                    const int8_t *__restrict__ code, int64_t nbc, int64_t nb,
                                                    double *__restrict__ A, int64_t lda)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bi = b / nbc, bj = b - (b / nbc) * nbc;
        int8_t c[kKeep];
        load_codes(code + b * kKeep, c);
        double out[64];
        decompress_block(__ldg(f + b), __ldg(s + b), __ldg(phi + b), c, out);
        double *p = A + (bi * 8) * lda + bj * 8;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (kVec) {
                double2 *q = reinterpret_cast<double2 *>(p + i * lda);
#pragma unroll
                for (int h = 0; h < 4; ++h) q[h] = make_double2(out[i * 8 + 2 * h], out[i * 8 + 2 * h + 1]);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) p[i * lda + j] = out[i * 8 + j];
            }
        }
    }
}

static int grid_for(int64_t nb, int threads)
{
    int64_t want = (nb + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 64;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

static bool vec_ok(const void *p, int64_t ld) { return ((uintptr_t)p % 16 == 0) && (ld % 2 == 0); }

int launch_compress(const double *A, int64_t lda, const blaz_cmat *out, cudaStream_t st)
{
    const int64_t nbc = out->cols / 8, nb = (out->rows / 8) * nbc;
    if (nb == 0) return BLAZ_OK;
    const int threads = 128;
    const int grid = grid_for(nb, threads);
    if (vec_ok(A, lda))
        k_compress<true><<<grid, threads, 0, st>>>(A, lda, nbc, nb, out->f, out->s, out->phi, out->code);
    else
        k_compress<false><<<grid, threads, 0, st>>>(A, lda, nbc, nb, out->f, out->s, out->phi, out->code);
    return launch_status();
}

int launch_decompress(const blaz_cmat *a, double *A, int64_t lda, cudaStream_t st)
{
    const int64_t nbc = a->cols / 8, nb = (a->rows / 8) * nbc;
    if (nb == 0) return BLAZ_OK;
    const int threads = 128;
    const int grid = grid_for(nb, threads);
    if (vec_ok(A, lda))
        k_decompress<true><<<grid, threads, 0, st>>>(a->f, a->s, a->phi, a->code, nbc, nb, A, lda);
    else
        k_decompress<false><<<grid, threads, 0, st>>>(a->f, a->s, a->phi, a->code, nbc, nb, A, lda);
    return launch_status();
}

}  // namespace blaz
