// block_ops.cuh -- per-block device code of the operations on compressed
// blocks, shared by the standalone kernels and the persistent batch kernel:
// addition / subtraction (Algorithm 1, Eq. eq55 of "Compressed Matrix
// Computations", arXiv 2202.13007) and multiplication by a constant
// (Algorithm 2).  Bit-exact binary64 (explicit round-to-nearest intrinsics).
#pragma once

#include "blaz_internal.cuh"

namespace blaz {

// Block b of out = a +- b.  Every input of the block is read before anything
// is written, so out may alias a or b.
template <bool kSub>
__device__ __forceinline__ void add_block(int64_t b, const double *f1, const double *s1, const uint8_t *p1,
                                          const int8_t *c1, const double *f2, const double *s2, const uint8_t *p2,
                                          const int8_t *c2, double *f, double *s, uint8_t *p, int8_t *c)
{
    const double fa = f1[b], fb = f2[b], sa = s1[b], sb = s2[b];
    const int pa = p1[b], pb = p2[b];
    uint32_t wa[7], wb[7];
    const uint32_t *ca = reinterpret_cast<const uint32_t *>(c1 + b * kKeep);
    const uint32_t *cb = reinterpret_cast<const uint32_t *>(c2 + b * kKeep);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        wa[q] = ca[q];
        wb[q] = cb[q];
    }
    const double fs = kSub ? dsub(fa, fb) : dadd(fa, fb);
    const double ss = dadd(sa, sb);
    int ph = (pa * pb) / (pa + pb);
    ph = ph < 1 ? 1 : ph;
    uint32_t wo[7];
    if (ss == 0.0) {
#pragma unroll
        for (int q = 0; q < 7; ++q) wo[q] = 0u;
    } else {
        const double a1 = ddiv(sa, ss);
        const double a2 = ddiv(sb, ss);
        const double b1 = dmul(ddiv(a1, (double)pa), (double)ph);
        const double b2 = dmul(ddiv(a2, (double)pb), (double)ph);
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            uint32_t v = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double x1 = (double)(int8_t)(uint8_t)(wa[q] >> (8 * k));
                const double x2 = (double)(int8_t)(uint8_t)(wb[q] >> (8 * k));
                const double y = kSub ? dsub(dmul(b1, x1), dmul(b2, x2)) : dadd(dmul(b1, x1), dmul(b2, x2));
                v |= (uint32_t)(uint8_t)quantize(y) << (8 * k);
            }
            wo[q] = v;
        }
    }
    f[b] = fs;
    s[b] = ss;
    p[b] = (uint8_t)ph;
    uint32_t *co = reinterpret_cast<uint32_t *>(c + b * kKeep);
#pragma unroll
    for (int q = 0; q < 7; ++q) co[q] = wo[q];
}

// Block b of out = cst * a (Algorithm 2); phi and codes copied when out != a.
__device__ __forceinline__ void scale_block(int64_t b, const double *f1, const double *s1, const uint8_t *p1,
                                            const int8_t *c1, double cst, double *f, double *s, uint8_t *p,
                                            int8_t *c, bool copy)
{
    f[b] = dmul(f1[b], cst);
    s[b] = dmul(s1[b], cst);
    if (copy) {
        p[b] = p1[b];
        const uint32_t *src = reinterpret_cast<const uint32_t *>(c1 + b * kKeep);
        uint32_t *dst = reinterpret_cast<uint32_t *>(c + b * kKeep);
#pragma unroll
        for (int q = 0; q < 7; ++q) dst[q] = src[q];
    }
}

}  // namespace blaz
