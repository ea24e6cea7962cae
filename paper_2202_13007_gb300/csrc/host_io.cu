// host_io.cu -- compressed-matrix operations on host buffers: compression
// of a matrix that lives in host memory, pipelined with its transfer, and
// the transfer of a compressed matrix (the 45-byte block payload of Sec. II
// of "Compressed Matrix Computations", arXiv 2202.13007) to and from host
// memory.
//
// The host-to-device link is the bound of compressing a host matrix (about
// 210 GB/s on this machine against ~700 GB/s of compression throughput), so
// the matrix is moved in slabs of block rows on a copy stream into a ring of
// device staging buffers (up to 512 MB, kept from call to call) while the
// caller's stream compresses the slabs already landed; every slab's blocks
// form a contiguous range of the output.
#include <mutex>
#include <vector>

#include "blaz_internal.cuh"

namespace blaz {
namespace {

// Target bytes per slab.  Each slab costs nine host calls (a copy, events,
// the compressor's memset and three launches); at 48 MB slabs a 2 GB matrix
// took 43 of them and 4-7 ms of host time per call, enough on a slow host to
// fall behind the copy engine (21-27 ms for a 4.3 GB step against a 20.3 ms
// copy); at 128 MB the host spends 0.16 ms per call and the step stays at
// 20.9 ms, the longer first slab being the only cost.
constexpr size_t kSlabBytes = (size_t)128 << 20;
// Staging in flight: up to 512 MB (four slabs), so that the transfer can run
// ~2.4 ms ahead of compressions queued behind other work on the caller's
// stream.
constexpr size_t kRingBytes = (size_t)512 << 20;
constexpr int kRingMax = 16;

// One non-blocking copy stream per device, shared by all calls so that the
// transfers of successive calls queue behind each other in issue order.
cudaStream_t copy_stream(int dev)
{
    static std::mutex mu;
    static std::vector<cudaStream_t> streams;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)streams.size() <= dev) streams.resize(dev + 1, nullptr);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
        streams[dev] = nullptr;
    return streams[dev];
}

// The staging ring of one device, kept from call to call.  Allocating a
// fresh ring per call made each call wait on the host (inside the
// stream-ordered allocation) for the previous call's ring to be released,
// i.e. for the previous transfer to end, so the next call's copies were
// issued late.  Buffer b of the ring is reused once the compression of its
// previous slab has passed `freed[b]`; `landed[b]` orders that compression
// after the copy.  Calls on one device issue under the ring's mutex.
struct Ring {
    std::mutex mu;
    char *base = nullptr;
    size_t bytes = 0;       // allocated
    size_t buf_bytes = 0;   // current partition
    int nbuf = 0, next = 0;
    bool used[kRingMax] = {};
    cudaEvent_t freed[kRingMax] = {}, landed[kRingMax] = {};
};

Ring &ring_of(int dev)
{
    static std::mutex mu;
    static std::vector<Ring *> rings;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)rings.size() <= dev) rings.resize(dev + 1, nullptr);
    if (!rings[dev]) rings[dev] = new Ring();  // lives until the process exits
    return *rings[dev];
}

// Makes `cs` wait until every buffer of the current partition is free.
cudaError_t ring_drain(Ring &r, cudaStream_t cs)
{
    for (int b = 0; b < r.nbuf; ++b)
        if (r.used[b]) {
            cudaError_t e = cudaStreamWaitEvent(cs, r.freed[b], 0);
            if (e != cudaSuccess) return e;
            r.used[b] = false;
        }
    return cudaSuccess;
}

// Partitions the ring into `nbuf` buffers of `buf_bytes`, growing the
// allocation (stream-ordered on the copy stream) when it is too small.
int ring_prepare(Ring &r, size_t buf_bytes, int nbuf, cudaStream_t cs)
{
    cudaError_t e;
    for (int b = 0; b < kRingMax; ++b)
        if (!r.freed[b]) {
            if ((e = cudaEventCreateWithFlags(&r.freed[b], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&r.landed[b], cudaEventDisableTiming)) != cudaSuccess)
                return set_cuda_error(e);
        }
    if (r.buf_bytes == buf_bytes && r.nbuf == nbuf && r.base) return BLAZ_OK;
    // a new partition: every buffer of the old one must be free first
    if ((e = ring_drain(r, cs)) != cudaSuccess) return set_cuda_error(e);
    const size_t need = buf_bytes * (size_t)nbuf;
    if (need > r.bytes) {
        if (r.base) cudaFreeAsync(r.base, cs);
        r.base = nullptr;
        r.bytes = 0;
        keep_pool_cached();
        void *p = nullptr;
        if ((e = cudaMallocAsync(&p, need, cs)) != cudaSuccess) {
            (void)cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? BLAZ_ERR_OOM : set_cuda_error(e);
        }
        r.base = (char *)p;
        r.bytes = need;
    }
    r.buf_bytes = buf_bytes;
    r.nbuf = nbuf;
    r.next = 0;
    return BLAZ_OK;
}

}  // namespace
}  // namespace blaz

using namespace blaz;

extern "C" {

int blaz_compress_host(const double *A, int64_t lda, blaz_cmat *out, void *stream)
{
    BLAZ_NVTX();
    int rc = validate_cmat(out);
    if (rc) return rc;
    const int64_t rows = out->rows, cols = out->cols, nbc = cols / 8;
    if (rows == 0 || cols == 0) return BLAZ_OK;
    if (!A) return BLAZ_ERR_NULL;
    if (lda < cols) return BLAZ_ERR_LD;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e);
    cudaStream_t cs = copy_stream(dev);
    if (!cs) return BLAZ_ERR_CUDA;

    const size_t row_bytes = sizeof(double) * (size_t)cols;
    int64_t slab = (int64_t)(kSlabBytes / row_bytes) / 8 * 8;
    if (slab < 8) slab = 8;
    if (slab > rows) slab = rows;
    const int64_t nslab = (rows + slab - 1) / slab;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t buf_bytes = up(row_bytes * (size_t)slab);
    int64_t ring = (int64_t)(kRingBytes / buf_bytes);
    ring = ring < 2 ? 2 : (ring > kRingMax ? kRingMax : ring);
    Scratch ws(st);  // compress lists, reused slab after slab on `st`
    if ((rc = ws.alloc(compress_scratch_bytes((slab / 8) * nbc)))) return rc;
    Ring &R = ring_of(dev);
    std::lock_guard<std::mutex> lk(R.mu);
    // keep the largest partition the ring has (fewer re-partitions for a
    // stream of smaller calls); grow it when this call needs more
    int nbuf = (int)(nslab < ring ? nslab : ring);
    if (R.base && R.buf_bytes >= buf_bytes && R.nbuf >= 2) nbuf = R.nbuf;
    const size_t bbytes = (R.base && R.buf_bytes >= buf_bytes && R.nbuf >= 2) ? R.buf_bytes : buf_bytes;
    if ((rc = ring_prepare(R, bbytes, nbuf, cs))) return rc;
    for (int64_t k = 0; k < nslab; ++k) {
        const int b = R.next;
        R.next = (R.next + 1) % R.nbuf;
        const int64_t r0 = k * slab, nr = rows - r0 < slab ? rows - r0 : slab;
        double *buf = (double *)(R.base + (size_t)b * R.buf_bytes);
        if (R.used[b] && (e = cudaStreamWaitEvent(cs, R.freed[b], 0)) != cudaSuccess) return set_cuda_error(e);
        // contiguous rows: one linear copy; otherwise a pitched copy
        e = lda == cols ? cudaMemcpyAsync(buf, A + r0 * lda, row_bytes * (size_t)nr, cudaMemcpyHostToDevice, cs)
                        : cudaMemcpy2DAsync(buf, row_bytes, A + r0 * lda, sizeof(double) * (size_t)lda, row_bytes,
                                            (size_t)nr, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(R.landed[b], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, R.landed[b], 0);
        if (e != cudaSuccess) return set_cuda_error(e);
        const int64_t b0 = (r0 / 8) * nbc;
        blaz_cmat sub{nr, cols, out->f + b0, out->s + b0, out->phi + b0, out->code + b0 * kKeep};
        if ((rc = launch_compress(buf, cols, nr, cols, &sub, ws.p, st))) return rc;
        if ((e = cudaEventRecord(R.freed[b], st)) != cudaSuccess) return set_cuda_error(e);
        R.used[b] = true;
    }
    return BLAZ_OK;
}

// Packed payload layout (as in a file): f[nb], s[nb] (binary64), phi[nb], code[nb][28].
static int payload_copy(const blaz_cmat *a, unsigned char *host, bool to_host, cudaStream_t st)
{
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    if (nb == 0) return BLAZ_OK;
    if (!host) return BLAZ_ERR_NULL;
    const size_t n8 = (size_t)nb * 8;
    const cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
    void *dev[4] = {a->f, a->s, a->phi, a->code};
    const size_t off[4] = {0, n8, 2 * n8, 2 * n8 + (size_t)nb}, len[4] = {n8, n8, (size_t)nb, (size_t)nb * kKeep};
    for (int i = 0; i < 4; ++i) {
        cudaError_t e = to_host ? cudaMemcpyAsync(host + off[i], dev[i], len[i], kind, st)
                                : cudaMemcpyAsync(dev[i], host + off[i], len[i], kind, st);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return BLAZ_OK;
}

int blaz_cmat_download(const blaz_cmat *a, void *host, void *stream)
{
    BLAZ_NVTX();
    int rc = validate_cmat(a);
    if (rc) return rc;
    return payload_copy(a, (unsigned char *)host, true, (cudaStream_t)stream);
}

int blaz_cmat_upload(const void *host, blaz_cmat *a, void *stream)
{
    BLAZ_NVTX();
    int rc = validate_cmat(a);
    if (rc) return rc;
    return payload_copy(a, (unsigned char *)const_cast<void *>(host), false, (cudaStream_t)stream);
}

}  // extern "C"
