// split_bf16.cuh -- the three-slice bf16 form of a binary64 value used by the
// split-precision matrix product ("Matrix multiplication", Sec. III of
// "Compressed Matrix Computations", arXiv 2202.13007; k_mm_bf16.cu).
#pragma once

#include <cuda_bf16.h>

namespace blaz {

// x ~ x1 + x2 + x3, each the bf16 rounding of the remainder (computed in
// fp32, where the remainders are exact).
__device__ __forceinline__ void split3(double x, __nv_bfloat16 &x1, __nv_bfloat16 &x2, __nv_bfloat16 &x3)
{
    const float xf = (float)x;
    x1 = __float2bfloat16_rn(xf);
    const float r1 = xf - __bfloat162float(x1);
    x2 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(x2);
    x3 = __float2bfloat16_rn(r2);
}

}  // namespace blaz
