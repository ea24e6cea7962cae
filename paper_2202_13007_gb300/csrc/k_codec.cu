// k_codec.cu -- compressor and decompressor kernels (Sec. II of "Compressed
// Matrix Computations", arXiv 2202.13007).
//
// Compression is bit-exact binary64: every operation is an explicit
// round-to-nearest intrinsic in the order fixed in include/blaz.h, so the
// result does not depend on -fmad or on the compiler's scheduling.  The
// compressor runs in two kernels: k_compress_fast decides every block it can
// certify (compress_fast.cuh) and lists the others; k_compress_fix
// recompresses the listed blocks with the exact binary64 path, densely (one
// listed block per thread), so the rare exact blocks cost no warp divergence.
#include "compress_fast.cuh"

namespace blaz {

template <bool kVec>
__global__ void __launch_bounds__(128)
    k_compress_fast(const double *__restrict__ A, int64_t lda, int64_t nbc, int64_t nb, double *__restrict__ f,
                    double *__restrict__ s, uint8_t *__restrict__ phi, int8_t *__restrict__ code,
                    unsigned *__restrict__ fix_list, unsigned *__restrict__ fix_count)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bi = b / nbc, bj = b - (b / nbc) * nbc;
        double d[64];
        load_block<kVec>(A, lda, bi, bj, d);
        f[b] = d[0];
        double sv;
        uint8_t ph;
        int8_t c[kKeep];
        const bool ok = compress_block_fast(d, sv, ph, c);
        s[b] = sv;
        if (ok) {
            phi[b] = ph;
            store_codes(code + b * kKeep, c);
        }
        // Append the blocks left undecided, one atomic per warp.
        const unsigned act = __activemask();
        const unsigned need = __ballot_sync(act, !ok);
        if (need) {
            const int lane = threadIdx.x & 31;
            const int leader = __ffs(need) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(fix_count, (unsigned)__popc(need));
            base = __shfl_sync(act, base, leader);
            if (!ok) fix_list[base + __popc(need & ((1u << lane) - 1u))] = (unsigned)b;
        }
    }
}

// The exact binary64 compressor (compress_block) on the listed blocks.
template <bool kVec>
__global__ void __launch_bounds__(128)
    k_compress_fix(const double *__restrict__ A, int64_t lda, int64_t nbc, const unsigned *__restrict__ fix_list,
                   const unsigned *__restrict__ fix_count, double *__restrict__ f, double *__restrict__ s,
                   uint8_t *__restrict__ phi, int8_t *__restrict__ code)
{
    const int64_t n = *fix_count;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = fix_list[q];
        const int64_t bi = b / nbc, bj = b - (b / nbc) * nbc;
        double d[64];
        load_block<kVec>(A, lda, bi, bj, d);
        f[b] = d[0];
        double sv;
        uint8_t ph;
        int8_t c[kKeep];
        compress_block(d, sv, ph, c);
        s[b] = sv;
        phi[b] = ph;
        store_codes(code + b * kKeep, c);
    }
}

template <bool kVec>
__global__ void __launch_bounds__(128) k_decompress(const double *__restrict__ f, const double *__restrict__ s,
                                                    const uint8_t *__restrict__ phi,
                                                    const int8_t *__restrict__ code, int64_t nbc, int64_t nb,
                                                    double *__restrict__ A, int64_t lda)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bi = b / nbc, bj = b - (b / nbc) * nbc;
        int8_t c[kKeep];
        load_codes(code + b * kKeep, c);
        double out[64];
        decompress_block(__ldg(f + b), __ldg(s + b), __ldg(phi + b), c, out);
        double *p = A + (bi * 8) * lda + bj * 8;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (kVec) {
                double2 *q = reinterpret_cast<double2 *>(p + i * lda);
#pragma unroll
                for (int h = 0; h < 4; ++h) q[h] = make_double2(out[i * 8 + 2 * h], out[i * 8 + 2 * h + 1]);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) p[i * lda + j] = out[i * 8 + j];
            }
        }
    }
}

static int grid_for(int64_t nb, int threads)
{
    int64_t want = (nb + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 64;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

static bool vec_ok(const void *p, int64_t ld) { return ((uintptr_t)p % 16 == 0) && (ld % 2 == 0); }

size_t compress_scratch_bytes(int64_t nb) { return ((size_t)nb * 4 + 255) / 256 * 256 + 256; }

int launch_compress(const double *A, int64_t lda, const blaz_cmat *out, void *scratch, cudaStream_t st)
{
    const int64_t nbc = out->cols / 8, nb = (out->rows / 8) * nbc;
    if (nb == 0) return BLAZ_OK;
    if (nb > 0xFFFFFFFFll) return BLAZ_ERR_SHAPE;
    unsigned *list = (unsigned *)scratch;
    unsigned *count = (unsigned *)((char *)scratch + compress_scratch_bytes(nb) - 256);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return set_cuda_error(e);
    const int threads = 128;
    const int grid = grid_for(nb, threads);
    const int fix_grid = num_sms() * 4;
    if (vec_ok(A, lda)) {
        k_compress_fast<true><<<grid, threads, 0, st>>>(A, lda, nbc, nb, out->f, out->s, out->phi, out->code, list, count);
        k_compress_fix<true><<<fix_grid, threads, 0, st>>>(A, lda, nbc, list, count, out->f, out->s, out->phi, out->code);
    } else {
        k_compress_fast<false><<<grid, threads, 0, st>>>(A, lda, nbc, nb, out->f, out->s, out->phi, out->code, list, count);
        k_compress_fix<false><<<fix_grid, threads, 0, st>>>(A, lda, nbc, list, count, out->f, out->s, out->phi, out->code);
    }
    return launch_status();
}

int launch_decompress(const blaz_cmat *a, double *A, int64_t lda, cudaStream_t st)
{
    const int64_t nbc = a->cols / 8, nb = (a->rows / 8) * nbc;
    if (nb == 0) return BLAZ_OK;
    const int threads = 128;
    const int grid = grid_for(nb, threads);
    if (vec_ok(A, lda))
        k_decompress<true><<<grid, threads, 0, st>>>(a->f, a->s, a->phi, a->code, nbc, nb, A, lda);
    else
        k_decompress<false><<<grid, threads, 0, st>>>(a->f, a->s, a->phi, a->code, nbc, nb, A, lda);
    return launch_status();
}

}  // namespace blaz
