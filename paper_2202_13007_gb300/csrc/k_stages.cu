// k_stages.cu -- blaz_debug_block_stages: every intermediate stage of the
// compression of one 8x8 block (Sec. II of "Compressed Matrix Computations",
// arXiv 2202.13007: Eq. eqnorm, Eqs. eqslope / eqslope2, Eq. eqpredict,
// Eq. eqdct, Eq. eqphi), computed by one GPU thread in the binary64
// operation order of the compressor (compress_block), for inspection.
#include "block_codec.cuh"

namespace blaz {

__global__ void k_block_stages(const double *__restrict__ M, blaz_block_stages *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double d[64];
#pragma unroll
    for (int p = 0; p < 64; ++p) d[p] = M[p];
    out->f = d[0];
    // Eq. eqnorm (in place, from the last element backwards)
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
    for (int p = 0; p < 64; ++p) {
        out->delta[p] = d[p];
        K += (d[p] != 0.0);
    }
    const double S = tree_sum_abs(d);
    out->K = K;
    out->sum_abs = S;
    double s = 0.0;
    if (K > 0) {
        s = ddiv(S, (double)K);
        const double r = ddiv(1.0, s);
#pragma unroll
        for (int p = 0; p < 64; ++p) d[p] = dmul(d[p], r);
    } else {
#pragma unroll
        for (int p = 0; p < 64; ++p) d[p] = 0.0;
    }
    out->s = s;
    // Eq. eqpredict: nearest of the 256 reference slopes lo + k step
    double smax = 0.0;
#pragma unroll
    for (int p = 0; p < 64; ++p) {
        out->dprime[p] = d[p];
        const double a = fabs(d[p]);
        smax = a > smax ? a : smax;
    }
    out->s_max = smax;
    const double lo = dsub(s, smax), step = ddiv(dmul(2.0, smax), 256.0);
#pragma unroll
    for (int p = 0; p < 64; ++p) {
        double k = 0.0;
        if (smax > 0.0) {
            k = floor(dadd(ddiv(dsub(d[p], lo), step), 0.5));
            k = k < 0.0 ? 0.0 : (k > 255.0 ? 255.0 : k);
        }
        out->psi[p] = (uint8_t)k;
    }
    // Eq. eqdct, all 64 coefficients: inner sums over v, outer sums over u,
    // then alpha_i alpha_j; products by cos(0) = 1 are exact and omitted.
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
            out->dct[i * 8 + j] = X;
            const double ax = fabs(X);
            m = (ax > m) ? ax : m;
        }
    }
    out->m = m;
    // Eq. eqphi and the kept codes
    const double q = ddiv(127.0, m);
    int phi;
    if (!(q < 255.0)) phi = 255;
    else {
        phi = __double2int_rz(q);
        phi = phi < 1 ? 1 : phi;
    }
    out->phi = (uint8_t)phi;
    const double phid = (double)phi;
#pragma unroll
    for (int t = 0; t < kKeep; ++t) out->code[t] = quantize(dmul(out->dct[kept_row(t) * 8 + kept_col(t)], phid));
}

}  // namespace blaz

using namespace blaz;

extern "C" int blaz_debug_block_stages(const double *M, blaz_block_stages *out, void *stream)
{
    BLAZ_NVTX();
    if (!M || !out) return BLAZ_ERR_NULL;
    k_block_stages<<<1, 32, 0, (cudaStream_t)stream>>>(M, out);
    return launch_status();
}
