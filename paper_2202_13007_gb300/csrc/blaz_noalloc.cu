// blaz_noalloc.cu -- blaz_dot_noalloc: the flattened dot product without any
// device allocation.
//
// Some callers cannot let a library allocate device memory: a framework or a
// serving runtime that owns every byte of HBM through its own allocator or a
// fixed budget, a process on a driver or device without stream-ordered
// allocation (memory pools), or a hot loop that must not risk an
// out-of-memory failure or an allocator stall halfway through a step.
// blaz_dot needs a little scratch (one partial sum per CTA and an arrival
// counter) and takes it from cudaMallocAsync; this entry point takes it from
// a fixed array in the library's own device memory instead.
#include <mutex>
#include <vector>

#include "blaz_internal.cuh"

namespace blaz {

// The static scratch holds one partial sum for each CTA of the largest grid
// the flattened dot launches (kDotMaxCtas), then the arrival counter.
constexpr size_t kNoAllocCounterOffset = kDotMaxCtas * sizeof(double);
constexpr size_t kNoAllocBytes = kNoAllocCounterOffset + 256;

// Scratch of blaz_dot_noalloc: [0, 8192) partial sums, then the 32-bit arrival
// counter.  Every GPU that loads the library holds these 8448 bytes until the
// process exits.  Host code must not use the symbol itself as a pointer (on
// the host it is only a stand-in); the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_dot_scratch[kNoAllocBytes];

// Device address of g_dot_scratch, looked up once per device with that
// device current.
static void *scratch_address(int &status)
{
    static std::mutex mu;
    static std::vector<void *> addr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        status = set_cuda_error(e);
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dot_scratch);
        if (e != cudaSuccess || !p) {
            status = set_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
            return nullptr;
        }
        addr[dev] = p;
    }
    status = BLAZ_OK;
    return addr[dev];
}

}  // namespace blaz

using namespace blaz;

extern "C" int blaz_dot_noalloc(const blaz_cmat *a, const blaz_cmat *b, double *result, void *stream)
{
    BLAZ_NVTX();
    // The same descriptor checks as blaz_dot: sides, block-count limits, NULL
    // arrays and alignment, so no launch ever sees an overflowing shape.
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(b))) return rc;
    if (a->rows != b->rows || a->cols != b->cols) return BLAZ_ERR_SHAPE;
    if (!result) return BLAZ_ERR_NULL;
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    // The launch needs one partial-sum slot per CTA.
    const int grid = dot_grid(nb);
    if (grid > kDotMaxCtas) return BLAZ_ERR_RANGE;
    int status = BLAZ_OK;
    char *base = (char *)scratch_address(status);
    if (!base) return status;
    double *partials = (double *)base;
    unsigned *counter = (unsigned *)(base + kNoAllocCounterOffset);
    cudaStream_t st = (cudaStream_t)stream;
    // The array keeps the previous call's contents: the counter must start at 0.
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return set_cuda_error(e);
    return launch_dot(a, b, result, partials, counter, grid, st);
}
