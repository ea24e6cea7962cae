// probe.cu -- a measurement probe for the benchmark: the binary64 issue rate
// of the device, the ceiling of the kernels here that are bound by binary64
// arithmetic (the compressor, the decompressor's final FMA).
#include "blaz_internal.cuh"

namespace blaz {

constexpr int kProbeMaxWarps = 32;  // warps per SM (one CTA per SM)
constexpr int kProbeChains = 4;     // independent dependency chains per thread

__global__ void __launch_bounds__(kProbeMaxWarps * 32) k_probe_fp64(double *out, int64_t iters, double c)
{
    double x[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) x[i] = threadIdx.x * 1e-3 + i;
    for (int64_t it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) x[i] = __dadd_rn(x[i], c);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) s += x[i];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace blaz

using namespace blaz;

extern "C" int blaz_probe_fp64_rate(int64_t iters, int warps_per_sm, double *out, int64_t out_len, int64_t *ops,
                                    void *stream)
{
    BLAZ_NVTX();
    if (!out || !ops) return BLAZ_ERR_NULL;
    if (warps_per_sm < 1 || warps_per_sm > kProbeMaxWarps || iters < 1 || iters > (1ll << 30)) return BLAZ_ERR_ARG;
    const int64_t threads = (int64_t)num_sms() * warps_per_sm * 32;
    if (out_len < threads) return BLAZ_ERR_ARG;
    k_probe_fp64<<<num_sms(), warps_per_sm * 32, 0, (cudaStream_t)stream>>>(out, iters, 1.0);
    *ops = threads * iters * kProbeChains;
    return launch_status();
}
