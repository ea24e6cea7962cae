// blaz_api.cu -- the extern "C" entry points declared in include/blaz.h:
// argument validation on the host, then stream-ordered kernel launches.
#include <cstdio>
#include <mutex>
#include <vector>

#include "blaz_internal.cuh"
#include "rate.cuh"

namespace blaz {

static thread_local int g_last_cuda = 0;

int set_cuda_error(cudaError_t e)
{
    g_last_cuda = (int)e;
    return BLAZ_ERR_CUDA;
}

int launch_status()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BLAZ_OK : set_cuda_error(e);
}

void keep_pool_cached()
{
    static std::mutex mu;
    static std::vector<char> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)done.size() <= dev) done.resize(dev + 1, 0);
    if (done[dev]) return;
    done[dev] = 1;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
            (void)cudaGetLastError();
    } else {
        (void)cudaGetLastError();
    }
}

int num_sms()
{
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (cache[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

static int check_dims(int64_t rows, int64_t cols)
{
    if (rows < 0 || cols < 0 || rows % 8 || cols % 8) return BLAZ_ERR_SHAPE;
    // sides up to 2^34 and up to 2^40 blocks (45 TB): the block count and the
    // byte sizes stay far from int64 overflow
    if (rows > ((int64_t)1 << 34) || cols > ((int64_t)1 << 34) || (rows / 8) * (cols / 8) > ((int64_t)1 << 40))
        return BLAZ_ERR_SHAPE;
    return BLAZ_OK;
}

static int64_t nblocks(const blaz_cmat *m) { return (m->rows / 8) * (m->cols / 8); }

// A compressed matrix descriptor is valid when its sides are multiples of 8
// and, unless it is empty, all four arrays are set.
int validate_cmat(const blaz_cmat *m)
{
    if (!m) return BLAZ_ERR_NULL;
    int rc = check_dims(m->rows, m->cols);
    if (rc) return rc;
    if (nblocks(m) > 0 && (!m->f || !m->s || !m->phi || !m->code)) return BLAZ_ERR_NULL;
    // f and s are read as binary64, the codes as 32-bit words.
    if ((uintptr_t)m->f % 8 || (uintptr_t)m->s % 8 || (uintptr_t)m->code % 4) return BLAZ_ERR_ARG;
    return BLAZ_OK;
}

static int same_shape(const blaz_cmat *a, const blaz_cmat *b)
{
    return (a->rows == b->rows && a->cols == b->cols) ? BLAZ_OK : BLAZ_ERR_SHAPE;
}

}  // namespace blaz

using namespace blaz;

extern "C" {

const char *blaz_strerror(int status)
{
    switch (status) {
    case BLAZ_OK: return "ok";
    case BLAZ_ERR_SHAPE: return "shape: sides must be non-negative multiples of 8 and operands must conform";
    case BLAZ_ERR_NULL: return "a required pointer is NULL";
    case BLAZ_ERR_LD: return "leading dimension smaller than the row length";
    case BLAZ_ERR_OOM: return "device allocation failed";
    case BLAZ_ERR_CUDA: return "CUDA runtime or launch error";
    case BLAZ_ERR_BUSY: return "no free slot";
    case BLAZ_ERR_TIMEOUT: return "bounded device wait ran out";
    case BLAZ_ERR_BUDGET: return "request exceeds the admission budget";
    case BLAZ_ERR_ARG: return "invalid argument";
    case BLAZ_ERR_RANGE: return "index out of range";
    case BLAZ_ERR_IO: return "file open, read or write failed";
    case BLAZ_ERR_FORMAT: return "not a compressed-matrix file of this format";
    default: return "unknown status";
    }
}

int blaz_last_cuda_error(void) { return g_last_cuda; }

int blaz_probe_bounded_wait(int64_t max_cycles, void *stream)
{
    return launch_probe_wait(max_cycles, (cudaStream_t)stream);
}

int blaz_device_status(void *stream)
{
    int a = device_status((cudaStream_t)stream);
    int b = batch_device_status();
    int c = ops_device_status();
    return a != BLAZ_OK ? a : b != BLAZ_OK ? b : c;
}

void blaz_constants(double cos_out[64], double aa_out[64], int32_t kept_out[56])
{
    for (int k = 0; k < 8; ++k)
        for (int x = 0; x < 8; ++x) {
            if (cos_out) cos_out[k * 8 + x] = cos_tab(k, x);
            if (aa_out) aa_out[k * 8 + x] = aa_tab(k, x);
        }
    if (kept_out)
        for (int t = 0; t < kKeep; ++t) {
            kept_out[2 * t] = kept_row(t);
            kept_out[2 * t + 1] = kept_col(t);
        }
}

static int cmat_alloc(blaz_cmat *m, int64_t rows, int64_t cols, int nkeep, void *stream)
{
    if (!m) return BLAZ_ERR_NULL;
    int rc = check_dims(rows, cols);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    m->rows = rows;
    m->cols = cols;
    m->f = m->s = nullptr;
    m->phi = nullptr;
    m->code = nullptr;
    const int64_t nb = nblocks(m);
    if (nb == 0) return BLAZ_OK;
    // One allocation: f | s | code | phi (each 256-byte aligned).
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t of = 0, os = up(of + 8 * nb), oc = up(os + 8 * nb), op = up(oc + (size_t)nkeep * nb);
    const size_t total = up(op + nb);
    void *base = nullptr;
    cudaError_t e = cudaMallocAsync(&base, total, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? BLAZ_ERR_OOM : set_cuda_error(e);
    }
    char *b = (char *)base;
    m->f = (double *)(b + of);
    m->s = (double *)(b + os);
    m->code = (int8_t *)(b + oc);
    m->phi = (uint8_t *)(b + op);
    return BLAZ_OK;
}

int blaz_cmat_alloc(blaz_cmat *m, int64_t rows, int64_t cols, void *stream)
{
    return cmat_alloc(m, rows, cols, kKeep, stream);
}

int blaz_keep_count(int r) { return (r >= 1 && r <= 8) ? 8 * r + (8 - r) * r : -1; }

int blaz_cmat_alloc_rate(blaz_cmat *m, int64_t rows, int64_t cols, int r, void *stream)
{
    if (blaz_keep_count(r) < 0) return BLAZ_ERR_ARG;
    return cmat_alloc(m, rows, cols, blaz_keep_count(r), stream);
}

int blaz_cmat_free(blaz_cmat *m, void *stream)
{
    if (!m) return BLAZ_ERR_NULL;
    if (m->f) {
        cudaError_t e = cudaFreeAsync(m->f, (cudaStream_t)stream);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    m->f = m->s = nullptr;
    m->phi = nullptr;
    m->code = nullptr;
    return BLAZ_OK;
}

int blaz_compress(const double *A, int64_t lda, blaz_cmat *out, void *stream)
{
    BLAZ_NVTX();
    int rc = validate_cmat(out);
    if (rc) return rc;
    if (nblocks(out) == 0) return BLAZ_OK;
    if (!A) return BLAZ_ERR_NULL;
    if (lda < out->cols) return BLAZ_ERR_LD;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch ws(st);
    if ((rc = ws.alloc(compress_scratch_bytes(nblocks(out))))) return rc;
    return launch_compress(A, lda, out->rows, out->cols, out, ws.p, st);
}

static int64_t ceil8(int64_t n) { return (n + 7) / 8 * 8; }

// A logical rows x cols shape whose edge-replicated extension is a's block grid.
static int check_logical(const blaz_cmat *a, int64_t rows, int64_t cols)
{
    if (rows < 0 || cols < 0 || ceil8(rows) != a->rows || ceil8(cols) != a->cols) return BLAZ_ERR_SHAPE;
    return BLAZ_OK;
}

int blaz_compress_padded(const double *A, int64_t lda, int64_t rows, int64_t cols, blaz_cmat *out, void *stream)
{
    BLAZ_NVTX();
    int rc;
    if ((rc = validate_cmat(out)) || (rc = check_logical(out, rows, cols))) return rc;
    if (nblocks(out) == 0) return BLAZ_OK;
    if (!A) return BLAZ_ERR_NULL;
    if (lda < cols) return BLAZ_ERR_LD;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch ws(st);
    if ((rc = ws.alloc(compress_scratch_bytes(nblocks(out))))) return rc;
    return launch_compress(A, lda, rows, cols, out, ws.p, st);
}

int blaz_decompress_padded(const blaz_cmat *a, int64_t rows, int64_t cols, double *A, int64_t lda, void *stream)
{
    BLAZ_NVTX();
    int rc;
    if ((rc = validate_cmat(a)) || (rc = check_logical(a, rows, cols))) return rc;
    if (nblocks(a) == 0) return BLAZ_OK;
    if (!A) return BLAZ_ERR_NULL;
    if (lda < cols) return BLAZ_ERR_LD;
    return launch_decompress(a, A, lda, (cudaStream_t)stream, rows, cols, false);
}

int blaz_decompress(const blaz_cmat *a, double *A, int64_t lda, void *stream)
{
    BLAZ_NVTX();
    int rc = validate_cmat(a);
    if (rc) return rc;
    if (nblocks(a) == 0) return BLAZ_OK;
    if (!A) return BLAZ_ERR_NULL;
    if (lda < a->cols) return BLAZ_ERR_LD;
    return launch_decompress(a, A, lda, (cudaStream_t)stream);
}

static int add_or_sub(const blaz_cmat *a, const blaz_cmat *b, blaz_cmat *out, bool sub, void *stream)
{
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(b)) || (rc = validate_cmat(out))) return rc;
    if ((rc = same_shape(a, b)) || (rc = same_shape(a, out))) return rc;
    return launch_add(a, b, out, sub, (cudaStream_t)stream);
}

int blaz_add(const blaz_cmat *a, const blaz_cmat *b, blaz_cmat *out, void *stream)
{
    BLAZ_NVTX();
    return add_or_sub(a, b, out, false, stream);
}

int blaz_sub(const blaz_cmat *a, const blaz_cmat *b, blaz_cmat *out, void *stream)
{
    BLAZ_NVTX();
    return add_or_sub(a, b, out, true, stream);
}

int blaz_scale(const blaz_cmat *a, double c, blaz_cmat *out, void *stream)
{
    BLAZ_NVTX();
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(out))) return rc;
    if ((rc = same_shape(a, out))) return rc;
    return launch_scale(a, c, out, (cudaStream_t)stream);
}

int blaz_compress_rate(const double *A, int64_t lda, int r, blaz_cmat *out, void *stream)
{
    BLAZ_NVTX();
    if (blaz_keep_count(r) < 0) return BLAZ_ERR_ARG;
    int rc = validate_cmat(out);
    if (rc) return rc;
    if (nblocks(out) == 0) return BLAZ_OK;
    if (!A) return BLAZ_ERR_NULL;
    if (lda < out->cols) return BLAZ_ERR_LD;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch ws(st);
    if ((rc = ws.alloc(compress_rate_scratch_bytes(nblocks(out))))) return rc;
    return launch_compress_rate(A, lda, out, r, ws.p, st);
}

int blaz_decompress_rate(const blaz_cmat *a, int r, double *A, int64_t lda, void *stream)
{
    BLAZ_NVTX();
    if (blaz_keep_count(r) < 0) return BLAZ_ERR_ARG;
    int rc = validate_cmat(a);
    if (rc) return rc;
    if (nblocks(a) == 0) return BLAZ_OK;
    if (!A) return BLAZ_ERR_NULL;
    if (lda < a->cols) return BLAZ_ERR_LD;
    return launch_decompress_rate(a, r, A, lda, (cudaStream_t)stream);
}

static int add_or_sub_rate(const blaz_cmat *a, const blaz_cmat *b, int r, blaz_cmat *out, bool sub, void *stream)
{
    if (blaz_keep_count(r) < 0) return BLAZ_ERR_ARG;
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(b)) || (rc = validate_cmat(out))) return rc;
    if ((rc = same_shape(a, b)) || (rc = same_shape(a, out))) return rc;
    return launch_add_rate(a, b, out, r, sub, (cudaStream_t)stream);
}

int blaz_add_rate(const blaz_cmat *a, const blaz_cmat *b, int r, blaz_cmat *out, void *stream)
{
    BLAZ_NVTX();
    return add_or_sub_rate(a, b, r, out, false, stream);
}

int blaz_sub_rate(const blaz_cmat *a, const blaz_cmat *b, int r, blaz_cmat *out, void *stream)
{
    BLAZ_NVTX();
    return add_or_sub_rate(a, b, r, out, true, stream);
}

int blaz_scale_rate(const blaz_cmat *a, double c, int r, blaz_cmat *out, void *stream)
{
    BLAZ_NVTX();
    if (blaz_keep_count(r) < 0) return BLAZ_ERR_ARG;
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(out))) return rc;
    if ((rc = same_shape(a, out))) return rc;
    return launch_scale_rate(a, c, out, r, (cudaStream_t)stream);
}

int blaz_dot_rate(const blaz_cmat *a, const blaz_cmat *b, int r, double *result, void *stream)
{
    BLAZ_NVTX();
    if (blaz_keep_count(r) < 0) return BLAZ_ERR_ARG;
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(b))) return rc;
    if ((rc = same_shape(a, b))) return rc;
    if (!result) return BLAZ_ERR_NULL;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = dot_rate_grid(nblocks(a));
    Scratch ws(st);
    if ((rc = ws.alloc(sizeof(double) * grid + 256))) return rc;
    double *partials = (double *)ws.p;
    unsigned *counter = (unsigned *)((char *)ws.p + ((sizeof(double) * grid + 255) & ~(size_t)255));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (nblocks(a) == 0) {
        e = cudaMemsetAsync(result, 0, sizeof(double), st);
        return e == cudaSuccess ? BLAZ_OK : set_cuda_error(e);
    }
    return launch_dot_rate(a, b, r, result, partials, counter, st);
}

int blaz_dot_rowcol_rate(const blaz_cmat *a, const blaz_cmat *b, int r, int64_t i, int64_t j, double *result,
                         void *stream)
{
    BLAZ_NVTX();
    if (blaz_keep_count(r) < 0) return BLAZ_ERR_ARG;
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(b))) return rc;
    if (a->cols != b->rows) return BLAZ_ERR_SHAPE;
    if (!result) return BLAZ_ERR_NULL;
    if (i < 0 || i >= a->rows || j < 0 || j >= b->cols) return BLAZ_ERR_RANGE;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = rowcol_rate_grid(a->cols / 8);
    Scratch ws(st);
    if ((rc = ws.alloc(sizeof(double) * grid + 256))) return rc;
    double *partials = (double *)ws.p;
    unsigned *counter = (unsigned *)((char *)ws.p + ((sizeof(double) * grid + 255) & ~(size_t)255));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return set_cuda_error(e);
    return launch_dot_rowcol_rate(a, b, r, i, j, result, partials, counter, st);
}

int blaz_matmul_rate(const blaz_cmat *a, int r, const double *B, int64_t ldb, int64_t m, double *C, int64_t ldc,
                     int mode, void *stream)
{
    BLAZ_NVTX();
    if (blaz_keep_count(r) < 0) return BLAZ_ERR_ARG;
    int rc;
    if ((rc = validate_cmat(a))) return rc;
    if (m < 0) return BLAZ_ERR_SHAPE;
    if (mode != BLAZ_MM_FP64 && mode != BLAZ_MM_SPLIT_BF16) return BLAZ_ERR_ARG;
    const int64_t n = a->rows, k = a->cols;
    if (n == 0 || m == 0) return BLAZ_OK;
    if (!C || (k > 0 && !B)) return BLAZ_ERR_NULL;
    if (ldc < m || (k > 0 && ldb < m)) return BLAZ_ERR_LD;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ah_bytes = (sizeof(double) * (size_t)(n * k) + 255) & ~(size_t)255;
    const size_t extra = mode == BLAZ_MM_SPLIT_BF16 ? split_bf16_scratch_bytes(n, k, m) : 0;
    Scratch ws(st);
    if ((rc = ws.alloc(ah_bytes + extra))) return rc;
    double *Ah = (double *)ws.p;
    if (k > 0 && (rc = launch_decompress_rate(a, r, Ah, k, st))) return rc;
    if (mode == BLAZ_MM_SPLIT_BF16)
        return launch_matmul_split_bf16(Ah, k, B, ldb, C, ldc, n, k, m, (char *)ws.p + ah_bytes, st);
    return launch_gemm_fp64(Ah, k, B, ldb, C, ldc, n, k, m, st);
}

int blaz_matmul_cc_rate(const blaz_cmat *a, const blaz_cmat *b, int r, double *C, int64_t ldc, int mode,
                        void *stream)
{
    BLAZ_NVTX();
    if (blaz_keep_count(r) < 0) return BLAZ_ERR_ARG;
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(b))) return rc;
    if (a->cols != b->rows) return BLAZ_ERR_SHAPE;
    if (mode != BLAZ_MM_FP64 && mode != BLAZ_MM_SPLIT_BF16) return BLAZ_ERR_ARG;
    const int64_t n = a->rows, k = a->cols, m = b->cols;
    if (n == 0 || m == 0) return BLAZ_OK;
    if (!C) return BLAZ_ERR_NULL;
    if (ldc < m) return BLAZ_ERR_LD;
    cudaStream_t st = (cudaStream_t)stream;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t ah_bytes = up(sizeof(double) * (size_t)(n * k)), bh_bytes = up(sizeof(double) * (size_t)(k * m));
    const size_t extra = mode == BLAZ_MM_SPLIT_BF16 ? split_bf16_scratch_bytes(n, k, m) : 0;
    Scratch ws(st);
    if ((rc = ws.alloc(ah_bytes + bh_bytes + extra))) return rc;
    double *Ah = (double *)ws.p, *Bh = (double *)((char *)ws.p + ah_bytes);
    if (k > 0 && (rc = launch_decompress_rate(a, r, Ah, k, st))) return rc;
    if (k > 0 && (rc = launch_decompress_rate(b, r, Bh, m, st))) return rc;
    if (mode == BLAZ_MM_SPLIT_BF16)
        return launch_matmul_split_bf16(Ah, k, Bh, m, C, ldc, n, k, m, (char *)ws.p + ah_bytes + bh_bytes, st);
    return launch_gemm_fp64(Ah, k, Bh, m, C, ldc, n, k, m, st);
}

int blaz_dot(const blaz_cmat *a, const blaz_cmat *b, double *result, void *stream)
{
    BLAZ_NVTX();
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(b))) return rc;
    if ((rc = same_shape(a, b))) return rc;
    if (!result) return BLAZ_ERR_NULL;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = dot_grid(nblocks(a));
    Scratch ws(st);
    if ((rc = ws.alloc(sizeof(double) * grid + 256))) return rc;
    double *partials = (double *)ws.p;
    unsigned *counter = (unsigned *)((char *)ws.p + ((sizeof(double) * grid + 255) & ~(size_t)255));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return set_cuda_error(e);
    return launch_dot(a, b, result, partials, counter, grid, st);
}

int blaz_dot_padded(const blaz_cmat *a, const blaz_cmat *b, int64_t rows, int64_t cols, double *result,
                    void *stream)
{
    BLAZ_NVTX();
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(b))) return rc;
    if ((rc = same_shape(a, b)) || (rc = check_logical(a, rows, cols))) return rc;
    if (!result) return BLAZ_ERR_NULL;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = dot_grid(nblocks(a));
    Scratch ws(st);
    if ((rc = ws.alloc(sizeof(double) * grid + 256))) return rc;
    double *partials = (double *)ws.p;
    unsigned *counter = (unsigned *)((char *)ws.p + ((sizeof(double) * grid + 255) & ~(size_t)255));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return set_cuda_error(e);
    return launch_dot(a, b, result, partials, counter, grid, st, rows, cols);
}

int blaz_dot_rowcol(const blaz_cmat *a, const blaz_cmat *b, int64_t i, int64_t j, double *result, void *stream)
{
    BLAZ_NVTX();
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(b))) return rc;
    if (a->cols != b->rows) return BLAZ_ERR_SHAPE;
    if (!result) return BLAZ_ERR_NULL;
    if (i < 0 || i >= a->rows || j < 0 || j >= b->cols) return BLAZ_ERR_RANGE;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = rowcol_grid(a->cols / 8);
    Scratch ws(st);
    if ((rc = ws.alloc(sizeof(double) * grid + 256))) return rc;
    double *partials = (double *)ws.p;
    unsigned *counter = (unsigned *)((char *)ws.p + ((sizeof(double) * grid + 255) & ~(size_t)255));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return set_cuda_error(e);
    return launch_dot_rowcol(a, b, i, j, result, partials, counter, st);
}

int blaz_matmul(const blaz_cmat *a, const double *B, int64_t ldb, int64_t m, double *C, int64_t ldc, int mode,
                void *stream)
{
    BLAZ_NVTX();
    int rc;
    if ((rc = validate_cmat(a))) return rc;
    if (m < 0) return BLAZ_ERR_SHAPE;
    if (mode != BLAZ_MM_FP64 && mode != BLAZ_MM_SPLIT_BF16) return BLAZ_ERR_ARG;
    const int64_t n = a->rows, k = a->cols;
    if (n == 0 || m == 0) return BLAZ_OK;
    if (!C || (k > 0 && !B)) return BLAZ_ERR_NULL;
    if (ldc < m || (k > 0 && ldb < m)) return BLAZ_ERR_LD;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch ws(st);
    if (mode == BLAZ_MM_SPLIT_BF16) {  // A's bf16 slices straight from the codes
        if ((rc = ws.alloc(split_bf16_scratch_bytes(n, k, m)))) return rc;
        return launch_matmul_split_bf16_cmat(a, B, ldb, C, ldc, m, ws.p, st);
    }
    if ((rc = ws.alloc(sizeof(double) * (size_t)(n * k)))) return rc;
    double *Ah = (double *)ws.p;
    if (k > 0 && (rc = launch_decompress(a, Ah, k, st))) return rc;
    return launch_gemm_fp64(Ah, k, B, ldb, C, ldc, n, k, m, st);
}

int blaz_matmul_cc(const blaz_cmat *a, const blaz_cmat *b, double *C, int64_t ldc, int mode, void *stream)
{
    BLAZ_NVTX();
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(b))) return rc;
    if (a->cols != b->rows) return BLAZ_ERR_SHAPE;
    if (mode != BLAZ_MM_FP64 && mode != BLAZ_MM_SPLIT_BF16) return BLAZ_ERR_ARG;
    const int64_t n = a->rows, k = a->cols, m = b->cols;
    if (n == 0 || m == 0) return BLAZ_OK;
    if (!C) return BLAZ_ERR_NULL;
    if (ldc < m) return BLAZ_ERR_LD;
    cudaStream_t st = (cudaStream_t)stream;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t ah_bytes = up(sizeof(double) * (size_t)(n * k)), bh_bytes = up(sizeof(double) * (size_t)(k * m));
    Scratch ws(st);
    if (mode == BLAZ_MM_SPLIT_BF16) {  // A's slices from its codes, B decoded once, then split
        if ((rc = ws.alloc(bh_bytes + split_bf16_scratch_bytes(n, k, m)))) return rc;
        double *Bh = (double *)ws.p;
        if (k > 0 && (rc = launch_decompress(b, Bh, m, st))) return rc;
        return launch_matmul_split_bf16_cmat(a, Bh, m, C, ldc, m, (char *)ws.p + bh_bytes, st);
    }
    if ((rc = ws.alloc(ah_bytes + bh_bytes))) return rc;
    double *Ah = (double *)ws.p, *Bh = (double *)((char *)ws.p + ah_bytes);
    if (k > 0 && (rc = launch_decompress(a, Ah, k, st))) return rc;
    if (k > 0 && (rc = launch_decompress(b, Bh, m, st))) return rc;
    return launch_gemm_fp64(Ah, k, Bh, m, C, ldc, n, k, m, st);
}

// Dense product of a zero-filled decoded Ah (n8 x k8) by B, for logical
// n x k x m: B is copied into a zero-padded k8 x m scratch when k8 != k, and
// the n8 x m result is cropped into C when n8 != n.
static int padded_gemm(const double *Ah, int64_t n, int64_t k, int64_t n8, int64_t k8, const double *B, int64_t ldb,
                       int64_t m, double *C, int64_t ldc, int mode, char *scratch, cudaStream_t st)
{
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const double *Bu = B;
    int64_t ldbu = ldb;
    cudaError_t e = cudaSuccess;
    if (k8 != k) {
        double *Bp = (double *)scratch;
        scratch += up(sizeof(double) * (size_t)(k8 * m));
        if (k > 0)
            e = cudaMemcpy2DAsync(Bp, sizeof(double) * m, B, sizeof(double) * ldb, sizeof(double) * m, k,
                                  cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(Bp + k * m, 0, sizeof(double) * (size_t)((k8 - k) * m), st);
        if (e != cudaSuccess) return set_cuda_error(e);
        Bu = Bp;
        ldbu = m;
    }
    double *Cu = C;
    int64_t ldcu = ldc;
    if (n8 != n) {
        Cu = (double *)scratch;
        scratch += up(sizeof(double) * (size_t)(n8 * m));
        ldcu = m;
    }
    int rc = mode == BLAZ_MM_SPLIT_BF16 ? launch_matmul_split_bf16(Ah, k8, Bu, ldbu, Cu, ldcu, n8, k8, m, scratch, st)
                                        : launch_gemm_fp64(Ah, k8, Bu, ldbu, Cu, ldcu, n8, k8, m, st);
    if (rc || n8 == n) return rc;
    e = cudaMemcpy2DAsync(C, sizeof(double) * ldc, Cu, sizeof(double) * m, sizeof(double) * m, n,
                          cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? BLAZ_OK : set_cuda_error(e);
}

static size_t padded_gemm_bytes(int64_t n, int64_t k, int64_t n8, int64_t k8, int64_t m, int mode)
{
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return (k8 != k ? up(sizeof(double) * (size_t)(k8 * m)) : 0) + (n8 != n ? up(sizeof(double) * (size_t)(n8 * m)) : 0) +
           (mode == BLAZ_MM_SPLIT_BF16 ? split_bf16_scratch_bytes(n8, k8, m) : 0);
}

int blaz_matmul_padded(const blaz_cmat *a, int64_t n, int64_t k, const double *B, int64_t ldb, int64_t m, double *C,
                       int64_t ldc, int mode, void *stream)
{
    BLAZ_NVTX();
    int rc;
    if ((rc = validate_cmat(a)) || (rc = check_logical(a, n, k))) return rc;
    if (m < 0) return BLAZ_ERR_SHAPE;
    if (mode != BLAZ_MM_FP64 && mode != BLAZ_MM_SPLIT_BF16) return BLAZ_ERR_ARG;
    if (n == 0 || m == 0) return BLAZ_OK;
    if (!C || (k > 0 && !B)) return BLAZ_ERR_NULL;
    if (ldc < m || (k > 0 && ldb < m)) return BLAZ_ERR_LD;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n8 = a->rows, k8 = a->cols;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t ah = up(sizeof(double) * (size_t)(n8 * k8));
    Scratch ws(st);
    if ((rc = ws.alloc(ah + padded_gemm_bytes(n, k, n8, k8, m, mode)))) return rc;
    double *Ah = (double *)ws.p;
    if (k8 > 0 && (rc = launch_decompress(a, Ah, k8, st, n, k, true))) return rc;
    return padded_gemm(Ah, n, k, n8, k8, B, ldb, m, C, ldc, mode, (char *)ws.p + ah, st);
}

int blaz_matmul_cc_padded(const blaz_cmat *a, const blaz_cmat *b, int64_t n, int64_t k, int64_t m, double *C,
                          int64_t ldc, int mode, void *stream)
{
    BLAZ_NVTX();
    int rc;
    if ((rc = validate_cmat(a)) || (rc = validate_cmat(b))) return rc;
    if ((rc = check_logical(a, n, k)) || (rc = check_logical(b, k, m))) return rc;
    if (mode != BLAZ_MM_FP64 && mode != BLAZ_MM_SPLIT_BF16) return BLAZ_ERR_ARG;
    if (n == 0 || m == 0) return BLAZ_OK;
    if (!C) return BLAZ_ERR_NULL;
    if (ldc < m) return BLAZ_ERR_LD;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n8 = a->rows, k8 = a->cols, m8 = b->cols;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t ah = up(sizeof(double) * (size_t)(n8 * k8)), bh = up(sizeof(double) * (size_t)(k8 * m8));
    // B_hat is decoded zero-filled at its full k8 x m8 grid, so the product
    // runs on k8 x m8 and only the n x m corner is kept.
    const size_t cbytes = (n8 != n || m8 != m) ? up(sizeof(double) * (size_t)(n8 * m8)) : 0;
    const size_t extra = mode == BLAZ_MM_SPLIT_BF16 ? split_bf16_scratch_bytes(n8, k8, m8) : 0;
    Scratch ws(st);
    if ((rc = ws.alloc(ah + bh + cbytes + extra))) return rc;
    double *Ah = (double *)ws.p, *Bh = (double *)((char *)ws.p + ah);
    if (k8 > 0 && (rc = launch_decompress(a, Ah, k8, st, n, k, true))) return rc;
    if (k8 > 0 && (rc = launch_decompress(b, Bh, m8, st, k, m, true))) return rc;
    double *Cu = cbytes ? (double *)((char *)ws.p + ah + bh) : C;
    const int64_t ldcu = cbytes ? m8 : ldc;
    char *sx = (char *)ws.p + ah + bh + cbytes;
    rc = mode == BLAZ_MM_SPLIT_BF16 ? launch_matmul_split_bf16(Ah, k8, Bh, m8, Cu, ldcu, n8, k8, m8, sx, st)
                                    : launch_gemm_fp64(Ah, k8, Bh, m8, Cu, ldcu, n8, k8, m8, st);
    if (rc || !cbytes) return rc;
    cudaError_t e = cudaMemcpy2DAsync(C, sizeof(double) * ldc, Cu, sizeof(double) * m8, sizeof(double) * m, n,
                                      cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? BLAZ_OK : set_cuda_error(e);
}

}  // extern "C"
