// const_upload.cuh -- host-computed constant tables (fixed-point slices of the
// decompression map and of its Gram form) placed in a __device__ variable
// once per device, so that kernels read them from global memory with
// coalesced loads: passed as a large kernel parameter or a __constant__
// array, the per-lane indexed copy into shared memory is served by the
// constant cache one address at a time.
#pragma once

#include <mutex>

#include "blaz_internal.cuh"

namespace blaz {

// Copies `bytes` of `host` to the device variable `symbol` (at `offset`) on
// `st` the first time it is called for the current device, and waits for the
// copy; later calls return at once.  The first call on a device must not be
// made while `st` is being captured into a graph (refused, BLAZ_ERR_CUDA).
struct DeviceTable {
    std::mutex mu;
    bool done[64] = {};

    int ensure(const void *symbol, const void *host, size_t bytes, size_t offset, cudaStream_t st)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return set_cuda_error(e);
        if (dev < 0 || dev >= 64) return BLAZ_ERR_ARG;
        std::lock_guard<std::mutex> lk(mu);
        if (done[dev]) return BLAZ_OK;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(st, &cs);
        if (e != cudaSuccess) return set_cuda_error(e);
        if (cs != cudaStreamCaptureStatusNone) return set_cuda_error(cudaErrorStreamCaptureUnsupported);
        e = cudaMemcpyToSymbolAsync(symbol, host, bytes, offset, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_cuda_error(e);
        done[dev] = true;
        return BLAZ_OK;
    }
};

}  // namespace blaz
