// gmap.cuh -- the linear map of decompression (inverse of Sec. II of
// "Compressed Matrix Computations", arXiv 2202.13007) as a fixed matrix.
//
// Decompression is linear in the codes: block = f 1 + (s/phi) G c, where
// column t of the 64 x 28 matrix G is the block that kept coefficient t alone
// produces (the inverse DCT of a unit coefficient, then the inverse of
// Eq. eqnorm with f = 0).  G is computed once on the host in long double from
// the definitions; kernels use exact fixed-point slices of it (or of G^T G).
#pragma once

#include "blaz_internal.cuh"

namespace blaz {

// G[p][t], p = 8*row + col of the block, t = kept code index.
const long double (*decompress_map())[kKeep];

// Exact int64 -> binary64 (|v| < 2^53 exact; larger values truncated to 53
// bits), built from the bit pattern without the FP64 conversion unit.
__device__ __forceinline__ double i64_to_double(long long v)
{
    if (v == 0) return 0.0;
    const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const int e = 63 - __clzll((long long)a);
    const unsigned long long m = e <= 52 ? (a << (52 - e)) : (a >> (e - 52));
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 1023) << 52) | (m & 0x000FFFFFFFFFFFFFull)));
}

// Largest |Y| of a decoder's slice assembly Y = sum_sl Y_sl 2^(bits (S-1-sl)),
// where each Y_sl sums `terms` products of a digit (|digit| <= 2^(bits-1): the
// first digit of a map entry scaled below 2^(bits-1), later digits rounded
// residuals) by a code (|code| <= 127).
constexpr unsigned long long slice_assembly_bound(int slices, int bits, int terms)
{
    unsigned long long geo = 0;
    for (int k = 0; k < slices; ++k) geo += 1ull << (bits * k);
    return (unsigned long long)terms * (1ull << (bits - 1)) * 127ull * geo;
}

// |v| < 2^62 -> binary64 with the significand truncated to 53 bits (exact for
// |v| < 2^53), on the integer pipe: normalize left by the leading-zero count,
// one fixed right shift puts the leading one on bit 52, where it carries into
// the exponent field (hence 1085 - lz rather than 1086 - lz).  The decoders'
// assembled sums stay far below 2^62 (slice_assembly_bound of their slices
// over at most 64 codes; each decoder checks its own with a static_assert).
__device__ __forceinline__ double dec_to_double(long long v)
{
    const unsigned long long sign = (unsigned long long)v & 0x8000000000000000ull;
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const int lz = __clzll((long long)a);
    const unsigned long long m = (a << (lz & 63)) >> 11;
    const unsigned long long bits = sign | (m + ((unsigned long long)(1085 - lz) << 52));
    return a ? __longlong_as_double((long long)bits) : 0.0;
}

// Integer-valued float with |x| < 2^22 -> int (exact), without a conversion instruction.
__device__ __forceinline__ int f2i_small(float x) { return __float_as_int(x + 12582912.0f) - 0x4B400000; }

}  // namespace blaz
