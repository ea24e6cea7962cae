// rate.cuh -- launchers of the tunable-rate kernels (k_rate.cu): the first r
// DCT rows and columns kept, r = 1..8 (checked by the caller), code arrays of
// nb x keep(r) bytes.
#pragma once

#include "blaz_internal.cuh"

namespace blaz {

__host__ __device__ constexpr int rate_keep(int r) { return 8 * r + (8 - r) * r; }

size_t compress_rate_scratch_bytes(int64_t nb);
int launch_compress_rate(const double *A, int64_t lda, const blaz_cmat *out, int r, void *scratch, cudaStream_t st);
int launch_decompress_rate(const blaz_cmat *a, int r, double *A, int64_t lda, cudaStream_t st);
int launch_add_rate(const blaz_cmat *a, const blaz_cmat *b, const blaz_cmat *out, int r, bool subtract,
                    cudaStream_t st);
int launch_scale_rate(const blaz_cmat *a, double c, const blaz_cmat *out, int r, cudaStream_t st);
// flattened dot (grid CTAs, one partial each) and Algorithm 3's line x column
int dot_rate_grid(int64_t nb);
int launch_dot_rate(const blaz_cmat *a, const blaz_cmat *b, int r, double *result, double *partials,
                    unsigned *counter, cudaStream_t st);
int rowcol_rate_grid(int64_t nkb);
int launch_dot_rowcol_rate(const blaz_cmat *a, const blaz_cmat *b, int r, int64_t i, int64_t j, double *result,
                           double *partials, unsigned *counter, cudaStream_t st);

}  // namespace blaz
