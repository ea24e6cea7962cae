// cmat_io.cu -- save and load compressed matrices (the 360-bit block payload
// of Sec. II of "Compressed Matrix Computations", arXiv 2202.13007, as a
// file).  Host-side and blocking; the layout is documented with the entry
// points in include/blaz.h.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "blaz_internal.cuh"

namespace blaz {
namespace {

constexpr char kMagic[8] = {'B', 'L', 'A', 'Z', 'C', 'M', 'A', 'T'};
constexpr uint32_t kVersion = 1, kHeaderBytes = 64;
constexpr uint64_t kBlockBytes = 8 + 8 + 1 + kKeep;  // f, s, phi, codes

struct Header {
    char magic[8];
    uint32_t version, header_bytes;
    int64_t rows, cols, nb;
    uint64_t payload_bytes, hash, zero;
};
static_assert(sizeof(Header) == kHeaderBytes, "header layout");

// FNV-1a, 64-bit (offset basis 14695981039346656037, prime 1099511628211),
// taken over the payload as little-endian 64-bit words (the last word padded
// with zero bytes) rather than bytes: eight times fewer steps.
uint64_t fnv1a64(const unsigned char *p, size_t n)
{
    uint64_t h = 14695981039346656037ull;
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
        uint64_t w;
        std::memcpy(&w, p + i, 8);
        h ^= w;
        h *= 1099511628211ull;
    }
    if (i < n) {
        uint64_t w = 0;
        std::memcpy(&w, p + i, n - i);
        h ^= w;
        h *= 1099511628211ull;
    }
    return h;
}

struct File {
    FILE *f = nullptr;
    File(const char *path, const char *mode) : f(std::fopen(path, mode)) {}
    ~File()
    {
        if (f) std::fclose(f);
    }
    bool close()
    {
        const bool ok = f && std::fclose(f) == 0;
        f = nullptr;
        return ok;
    }
};

bool valid_shape(int64_t rows, int64_t cols)
{
    return rows >= 0 && cols >= 0 && rows % 8 == 0 && cols % 8 == 0 && rows <= (int64_t)1 << 40 &&
           cols <= (int64_t)1 << 40 && (rows / 8) * (cols / 8) <= ((int64_t)1 << 40);
}

// Reads and checks the header; the file position is left at the payload.
int read_header(FILE *f, Header &h)
{
    if (std::fread(&h, sizeof(h), 1, f) != 1) return BLAZ_ERR_FORMAT;
    if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion || h.header_bytes != kHeaderBytes ||
        h.zero != 0)
        return BLAZ_ERR_FORMAT;
    if (!valid_shape(h.rows, h.cols) || h.nb != (h.rows / 8) * (h.cols / 8) ||
        h.payload_bytes != (uint64_t)h.nb * kBlockBytes)
        return BLAZ_ERR_FORMAT;
    return BLAZ_OK;
}

}  // namespace
}  // namespace blaz

using namespace blaz;

extern "C" {

int blaz_cmat_save(const blaz_cmat *a, const char *path, void *stream)
{
    BLAZ_NVTX();
    int rc;
    if (!path) return BLAZ_ERR_NULL;
    if ((rc = validate_cmat(a))) return rc;
    const int64_t nb = (a->rows / 8) * (a->cols / 8);
    std::vector<unsigned char> payload((size_t)nb * kBlockBytes);
    cudaStream_t st = (cudaStream_t)stream;
    if (nb > 0) {
        unsigned char *p = payload.data();
        const size_t n8 = (size_t)nb * 8;
        cudaError_t e = cudaMemcpyAsync(p, a->f, n8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p + n8, a->s, n8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p + 2 * n8, a->phi, (size_t)nb, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p + 2 * n8 + nb, a->code, (size_t)nb * kKeep, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    Header h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.header_bytes = kHeaderBytes;
    h.rows = a->rows;
    h.cols = a->cols;
    h.nb = nb;
    h.payload_bytes = payload.size();
    h.hash = fnv1a64(payload.data(), payload.size());
    h.zero = 0;
    const std::string tmp = std::string(path) + ".tmp";
    {
        File f(tmp.c_str(), "wb");
        if (!f.f) return BLAZ_ERR_IO;
        bool ok = std::fwrite(&h, sizeof(h), 1, f.f) == 1;
        if (ok && !payload.empty()) ok = std::fwrite(payload.data(), payload.size(), 1, f.f) == 1;
        ok = f.close() && ok;
        if (!ok) {
            std::remove(tmp.c_str());
            return BLAZ_ERR_IO;
        }
    }
    if (std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return BLAZ_ERR_IO;
    }
    return BLAZ_OK;
}

int blaz_cmat_file_info(const char *path, int64_t *rows, int64_t *cols)
{
    if (!path || !rows || !cols) return BLAZ_ERR_NULL;
    File f(path, "rb");
    if (!f.f) return BLAZ_ERR_IO;
    Header h;
    int rc = read_header(f.f, h);
    if (rc) return rc;
    *rows = h.rows;
    *cols = h.cols;
    return BLAZ_OK;
}

int blaz_cmat_load(const char *path, blaz_cmat *out, void *stream)
{
    BLAZ_NVTX();
    if (!path || !out) return BLAZ_ERR_NULL;
    File f(path, "rb");
    if (!f.f) return BLAZ_ERR_IO;
    Header h;
    int rc = read_header(f.f, h);
    if (rc) return rc;
    std::vector<unsigned char> payload((size_t)h.payload_bytes);
    if (!payload.empty() && std::fread(payload.data(), payload.size(), 1, f.f) != 1) return BLAZ_ERR_FORMAT;
    if (std::fgetc(f.f) != EOF) return BLAZ_ERR_FORMAT;  // trailing bytes
    if (fnv1a64(payload.data(), payload.size()) != h.hash) return BLAZ_ERR_FORMAT;
    if (out->rows != h.rows || out->cols != h.cols) return BLAZ_ERR_SHAPE;
    if ((rc = validate_cmat(out))) return rc;
    const int64_t nb = h.nb;
    if (nb == 0) return BLAZ_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned char *p = payload.data();
    const size_t n8 = (size_t)nb * 8;
    cudaError_t e = cudaMemcpyAsync(out->f, p, n8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->s, p + n8, n8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->phi, p + 2 * n8, (size_t)nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out->code, p + 2 * n8 + nb, (size_t)nb * kKeep, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host payload is freed on return
    return e == cudaSuccess ? BLAZ_OK : set_cuda_error(e);
}

}  // extern "C"
