// exact_div.cuh -- correctly rounded binary64 division by a small positive
// integer without a division sequence, used where the specification of
// "Compressed Matrix Computations" (arXiv 2202.13007) divides by an integer:
// s = S/K (Eqs. eqslope, eqslope2) and a_k / phi_k in Algorithm 1.
//
// With y = RN(1/k), q = RN(x y) is within one ulp of x/k and the remainder
// r = x - k q is exact, so RN(q + r y) is the correctly rounded quotient
// (Markstein's theorem).  x/k is never a tie for an integer k (an odd k >= 3
// would need a 55-bit significand), so round-to-nearest-even is reached.  The
// argument keeps both steps in the normal range for 2^-900 <= |x| < Inf;
// other x take the general division.
#pragma once

#include "blaz_internal.cuh"
#include "gmap.cuh"

namespace blaz {

// RN(1/k) for k = 1..256 (entry k-1), exact hex literals.
__device__ __align__(16) double c_rcp_k[256] = {
    0x1.0000000000000p+0, 0x1.0000000000000p-1, 0x1.5555555555555p-2, 0x1.0000000000000p-2,
    0x1.999999999999ap-3, 0x1.5555555555555p-3, 0x1.2492492492492p-3, 0x1.0000000000000p-3,
    0x1.c71c71c71c71cp-4, 0x1.999999999999ap-4, 0x1.745d1745d1746p-4, 0x1.5555555555555p-4,
    0x1.3b13b13b13b14p-4, 0x1.2492492492492p-4, 0x1.1111111111111p-4, 0x1.0000000000000p-4,
    0x1.e1e1e1e1e1e1ep-5, 0x1.c71c71c71c71cp-5, 0x1.af286bca1af28p-5, 0x1.999999999999ap-5,
    0x1.8618618618618p-5, 0x1.745d1745d1746p-5, 0x1.642c8590b2164p-5, 0x1.5555555555555p-5,
    0x1.47ae147ae147bp-5, 0x1.3b13b13b13b14p-5, 0x1.2f684bda12f68p-5, 0x1.2492492492492p-5,
    0x1.1a7b9611a7b96p-5, 0x1.1111111111111p-5, 0x1.0842108421084p-5, 0x1.0000000000000p-5,
    0x1.f07c1f07c1f08p-6, 0x1.e1e1e1e1e1e1ep-6, 0x1.d41d41d41d41dp-6, 0x1.c71c71c71c71cp-6,
    0x1.bacf914c1bad0p-6, 0x1.af286bca1af28p-6, 0x1.a41a41a41a41ap-6, 0x1.999999999999ap-6,
    0x1.8f9c18f9c18fap-6, 0x1.8618618618618p-6, 0x1.7d05f417d05f4p-6, 0x1.745d1745d1746p-6,
    0x1.6c16c16c16c17p-6, 0x1.642c8590b2164p-6, 0x1.5c9882b931057p-6, 0x1.5555555555555p-6,
    0x1.4e5e0a72f0539p-6, 0x1.47ae147ae147bp-6, 0x1.4141414141414p-6, 0x1.3b13b13b13b14p-6,
    0x1.3521cfb2b78c1p-6, 0x1.2f684bda12f68p-6, 0x1.29e4129e4129ep-6, 0x1.2492492492492p-6,
    0x1.1f7047dc11f70p-6, 0x1.1a7b9611a7b96p-6, 0x1.15b1e5f75270dp-6, 0x1.1111111111111p-6,
    0x1.0c9714fbcda3bp-6, 0x1.0842108421084p-6, 0x1.0410410410410p-6, 0x1.0000000000000p-6,
    0x1.f81f81f81f820p-7, 0x1.f07c1f07c1f08p-7, 0x1.e9131abf0b767p-7, 0x1.e1e1e1e1e1e1ep-7,
    0x1.dae6076b981dbp-7, 0x1.d41d41d41d41dp-7, 0x1.cd85689039b0bp-7, 0x1.c71c71c71c71cp-7,
    0x1.c0e070381c0e0p-7, 0x1.bacf914c1bad0p-7, 0x1.b4e81b4e81b4fp-7, 0x1.af286bca1af28p-7,
    0x1.a98ef606a63bep-7, 0x1.a41a41a41a41ap-7, 0x1.9ec8e951033d9p-7, 0x1.999999999999ap-7,
    0x1.948b0fcd6e9e0p-7, 0x1.8f9c18f9c18fap-7, 0x1.8acb90f6bf3aap-7, 0x1.8618618618618p-7,
    0x1.8181818181818p-7, 0x1.7d05f417d05f4p-7, 0x1.78a4c8178a4c8p-7, 0x1.745d1745d1746p-7,
    0x1.702e05c0b8170p-7, 0x1.6c16c16c16c17p-7, 0x1.6816816816817p-7, 0x1.642c8590b2164p-7,
    0x1.6058160581606p-7, 0x1.5c9882b931057p-7, 0x1.58ed2308158edp-7, 0x1.5555555555555p-7,
    0x1.51d07eae2f815p-7, 0x1.4e5e0a72f0539p-7, 0x1.4afd6a052bf5bp-7, 0x1.47ae147ae147bp-7,
    0x1.446f86562d9fbp-7, 0x1.4141414141414p-7, 0x1.3e22cbce4a902p-7, 0x1.3b13b13b13b14p-7,
    0x1.3813813813814p-7, 0x1.3521cfb2b78c1p-7, 0x1.323e34a2b10bfp-7, 0x1.2f684bda12f68p-7,
    0x1.2c9fb4d812ca0p-7, 0x1.29e4129e4129ep-7, 0x1.27350b8812735p-7, 0x1.2492492492492p-7,
    0x1.21fb78121fb78p-7, 0x1.1f7047dc11f70p-7, 0x1.1cf06ada2811dp-7, 0x1.1a7b9611a7b96p-7,
    0x1.1811811811812p-7, 0x1.15b1e5f75270dp-7, 0x1.135c81135c811p-7, 0x1.1111111111111p-7,
    0x1.0ecf56be69c90p-7, 0x1.0c9714fbcda3bp-7, 0x1.0a6810a6810a7p-7, 0x1.0842108421084p-7,
    0x1.0624dd2f1a9fcp-7, 0x1.0410410410410p-7, 0x1.0204081020408p-7, 0x1.0000000000000p-7,
    0x1.fc07f01fc07f0p-8, 0x1.f81f81f81f820p-8, 0x1.f44659e4a4271p-8, 0x1.f07c1f07c1f08p-8,
    0x1.ecc07b301ecc0p-8, 0x1.e9131abf0b767p-8, 0x1.e573ac901e574p-8, 0x1.e1e1e1e1e1e1ep-8,
    0x1.de5d6e3f8868ap-8, 0x1.dae6076b981dbp-8, 0x1.d77b654b82c34p-8, 0x1.d41d41d41d41dp-8,
    0x1.d0cb58f6ec074p-8, 0x1.cd85689039b0bp-8, 0x1.ca4b3055ee191p-8, 0x1.c71c71c71c71cp-8,
    0x1.c3f8f01c3f8f0p-8, 0x1.c0e070381c0e0p-8, 0x1.bdd2b899406f7p-8, 0x1.bacf914c1bad0p-8,
    0x1.b7d6c3dda338bp-8, 0x1.b4e81b4e81b4fp-8, 0x1.b2036406c80d9p-8, 0x1.af286bca1af28p-8,
    0x1.ac5701ac5701bp-8, 0x1.a98ef606a63bep-8, 0x1.a6d01a6d01a6dp-8, 0x1.a41a41a41a41ap-8,
    0x1.a16d3f97a4b02p-8, 0x1.9ec8e951033d9p-8, 0x1.9c2d14ee4a102p-8, 0x1.999999999999ap-8,
    0x1.970e4f80cb872p-8, 0x1.948b0fcd6e9e0p-8, 0x1.920fb49d0e229p-8, 0x1.8f9c18f9c18fap-8,
    0x1.8d3018d3018d3p-8, 0x1.8acb90f6bf3aap-8, 0x1.886e5f0abb04ap-8, 0x1.8618618618618p-8,
    0x1.83c977ab2beddp-8, 0x1.8181818181818p-8, 0x1.7f405fd017f40p-8, 0x1.7d05f417d05f4p-8,
    0x1.7ad2208e0ecc3p-8, 0x1.78a4c8178a4c8p-8, 0x1.767dce434a9b1p-8, 0x1.745d1745d1746p-8,
    0x1.724287f46debcp-8, 0x1.702e05c0b8170p-8, 0x1.6e1f76b4337c7p-8, 0x1.6c16c16c16c17p-8,
    0x1.6a13cd1537290p-8, 0x1.6816816816817p-8, 0x1.661ec6a5122f9p-8, 0x1.642c8590b2164p-8,
    0x1.623fa77016240p-8, 0x1.6058160581606p-8, 0x1.5e75bb8d015e7p-8, 0x1.5c9882b931057p-8,
    0x1.5ac056b015ac0p-8, 0x1.58ed2308158edp-8, 0x1.571ed3c506b3ap-8, 0x1.5555555555555p-8,
    0x1.5390948f40febp-8, 0x1.51d07eae2f815p-8, 0x1.5015015015015p-8, 0x1.4e5e0a72f0539p-8,
    0x1.4cab88725af6ep-8, 0x1.4afd6a052bf5bp-8, 0x1.49539e3b2d067p-8, 0x1.47ae147ae147bp-8,
    0x1.460cbc7f5cf9ap-8, 0x1.446f86562d9fbp-8, 0x1.42d6625d51f87p-8, 0x1.4141414141414p-8,
    0x1.3fb013fb013fbp-8, 0x1.3e22cbce4a902p-8, 0x1.3c995a47babe7p-8, 0x1.3b13b13b13b14p-8,
    0x1.3991c2c187f63p-8, 0x1.3813813813814p-8, 0x1.3698df3de0748p-8, 0x1.3521cfb2b78c1p-8,
    0x1.33ae45b57bcb2p-8, 0x1.323e34a2b10bfp-8, 0x1.30d190130d190p-8, 0x1.2f684bda12f68p-8,
    0x1.2e025c04b8097p-8, 0x1.2c9fb4d812ca0p-8, 0x1.2b404ad012b40p-8, 0x1.29e4129e4129ep-8,
    0x1.288b01288b013p-8, 0x1.27350b8812735p-8, 0x1.25e22708092f1p-8, 0x1.2492492492492p-8,
    0x1.23456789abcdfp-8, 0x1.21fb78121fb78p-8, 0x1.20b470c67c0d9p-8, 0x1.1f7047dc11f70p-8,
    0x1.1e2ef3b3fb874p-8, 0x1.1cf06ada2811dp-8, 0x1.1bb4a4046ed29p-8, 0x1.1a7b9611a7b96p-8,
    0x1.19453808ca29cp-8, 0x1.1811811811812p-8, 0x1.16e0689427379p-8, 0x1.15b1e5f75270dp-8,
    0x1.1485f0e0acd3bp-8, 0x1.135c81135c811p-8, 0x1.12358e75d3033p-8, 0x1.1111111111111p-8,
    0x1.0fef010fef011p-8, 0x1.0ecf56be69c90p-8, 0x1.0db20a88f4696p-8, 0x1.0c9714fbcda3bp-8,
    0x1.0b7e6ec259dc8p-8, 0x1.0a6810a6810a7p-8, 0x1.0953f39010954p-8, 0x1.0842108421084p-8,
    0x1.073260a47f7c6p-8, 0x1.0624dd2f1a9fcp-8, 0x1.05197f7d73404p-8, 0x1.0410410410410p-8,
    0x1.03091b51f5e1ap-8, 0x1.0204081020408p-8, 0x1.0101010101010p-8, 0x1.0000000000000p-8};

// RN(x / k) for 1 <= k <= 256 (the general division for other k).
__device__ __forceinline__ double div_small_int(double x, int k)
{
    const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7FF;
    const double kd = i64_to_double(k);
    if (ex < 1023 - 900 || ex == 0x7FF || k < 1 || k > 256) return ddiv(x, kd);
    const double y = __ldg(&c_rcp_k[k - 1]);
    const double q = dmul(x, y);
    const double r = __fma_rn(-q, kd, x);
    return __fma_rn(r, y, q);
}

}  // namespace blaz
