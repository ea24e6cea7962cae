/*
 * blaz.h -- C ABI of the GB300 (sm_103a) implementation of the blaz
 * compressed-matrix method of "Compressed Matrix Computations"
 * (M. Martel, arXiv 2202.13007).
 *
 * A binary64 matrix whose sides are multiples of 8 is cut into 8x8 blocks
 * (Sec. II, "Block Splitting").  Each block is stored as
 *     f    binary64  first element M00                      (Sec. II, Eq. eqnorm)
 *     s    binary64  mean slope of the normalized block      (Eq. eqslope)
 *     phi  uint8     re-scaling factor 127/m, truncated      (Eq. eqphi)
 *     code int8[28]  truncated phi*DCT coefficients of the first two rows
 *                    and first two columns                   (Sec. II, Ex. 5)
 * i.e. 360 bits per block instead of 4096 (compression ratio 11.37).
 *
 * Conventions for every entry point below:
 *   - Matrices are row-major; lda/ldb/ldc are leading dimensions in elements.
 *   - Blocks are numbered row-major over the (rows/8) x (cols/8) block grid;
 *     kept code t of a block sits at code[block*28 + t], in the order
 *     row 0 (j = 0..7), row 1 (j = 0..7), then (i,0),(i,1) for i = 2..7.
 *   - Every pointer marked "device" must point to memory of the current CUDA
 *     device; "host" pointers are ordinary host memory.  The caller owns all
 *     buffers and streams it passes; the library keeps no reference to them
 *     after the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All work is enqueued asynchronously on it in stream order;
 *     the functions do not synchronize unless stated.
 *   - Return value: BLAZ_OK (0) or a negative BLAZ_ERR_* code.  Argument
 *     errors are detected on the host before anything is enqueued; a CUDA
 *     launch error is reported as BLAZ_ERR_CUDA (blaz_last_cuda_error() gives
 *     the CUDA error code).
 */
#ifndef BLAZ_H
#define BLAZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BLAZ_NKEEP 28

enum {
    BLAZ_OK = 0,
    BLAZ_ERR_SHAPE = -1,    /* a side is negative or not a multiple of 8, or shapes differ */
    BLAZ_ERR_NULL = -2,     /* a required pointer is NULL                                  */
    BLAZ_ERR_LD = -3,       /* leading dimension smaller than the row length               */
    BLAZ_ERR_OOM = -4,      /* device allocation failed                                    */
    BLAZ_ERR_CUDA = -5,     /* a CUDA runtime call or kernel launch failed                 */
    BLAZ_ERR_BUSY = -6,     /* server: no free slot right now                              */
    BLAZ_ERR_TIMEOUT = -7,  /* a bounded device wait ran out                               */
    BLAZ_ERR_BUDGET = -8,   /* server: request exceeds the admission budget                */
    BLAZ_ERR_ARG = -9,      /* any other invalid argument (mode, index, count)             */
    BLAZ_ERR_RANGE = -10,   /* an index is outside the matrix                              */
    BLAZ_ERR_IO = -11,      /* a file could not be opened, read or written                 */
    BLAZ_ERR_FORMAT = -12   /* a file is not a compressed matrix of this format            */
};

/* A compressed matrix: structure of arrays in device memory, nb = (rows/8)*(cols/8).
 * f and s must be 8-byte aligned and code 4-byte aligned (BLAZ_ERR_ARG otherwise). */
typedef struct blaz_cmat {
    int64_t rows, cols;   /* multiples of 8                               */
    double *f;            /* device, [nb]                                 */
    double *s;            /* device, [nb]                                 */
    uint8_t *phi;         /* device, [nb]                                 */
    int8_t *code;         /* device, [nb][28]                             */
} blaz_cmat;

/* Constant tables.  The first call on a device of an entry point that
 * decompresses (blaz_decompress*, blaz_matmul*) or takes a dot product
 * (blaz_dot*) copies the library's
 * fixed tables for it (slices of the decompression map, at most 44 KB) to
 * that device on `stream` and waits for the copy; later calls do not.  Make
 * that first call outside stream capture: during capture it is refused
 * (BLAZ_ERR_CUDA, cudaErrorStreamCaptureUnsupported). */

/* Human-readable name of a status code (static string). */
const char *blaz_strerror(int status);
/* CUDA error code (cudaError_t as int) of the last BLAZ_ERR_CUDA on this thread. */
int blaz_last_cuda_error(void);

/* Status of the library's kernels on the current device: synchronizes
 * `stream`, then returns BLAZ_ERR_TIMEOUT if a kernel's bounded wait ran out
 * since the last call (and clears the flag), else BLAZ_OK.  Kernels that wait
 * on barriers (the tensor-core product) give up after about two seconds
 * instead of hanging, record the timeout here and return. */
int blaz_device_status(void *stream);
/* Self-test of the device-side timeout path: one GPU thread waits on
 * `stream` for a device flag that nothing sets, for at most max_cycles SM
 * clock cycles (0 .. 4e9, else BLAZ_ERR_ARG), then records BLAZ_ERR_TIMEOUT in
 * the device status word (read and cleared by blaz_device_status) and
 * returns.  Every wait in the library's kernels is bounded the same way. */
int blaz_probe_bounded_wait(int64_t max_cycles, void *stream);
/* Measurement probe (no counterpart in the paper): one CTA of
 * 32 x warps_per_sm threads per SM (1 <= warps_per_sm <= 32, else
 * BLAZ_ERR_ARG) runs `iters` rounds of 4 independent binary64 additions per
 * thread on `stream`, writing one double per thread to out (device, out_len
 * >= 32 x warps_per_sm x SM count, else BLAZ_ERR_ARG; 1 <= iters <= 2^30).
 * *ops (host) gets the number of binary64 additions launched; their count
 * over the launch's duration is the device's binary64 issue rate at that
 * many warps per SM, whose maximum is the peak of the kernels bound by
 * binary64 arithmetic. */
int blaz_probe_fp64_rate(int64_t iters, int warps_per_sm, double *out, int64_t out_len, int64_t *ops,
                         void *stream);

/* Library-owned storage for a compressed matrix (stream-ordered allocation
 * on `stream`).  rows, cols >= 0 and multiples of 8.  The arrays are not
 * initialised.  Free with blaz_cmat_free on a stream ordered after last use. */
int blaz_cmat_alloc(blaz_cmat *m, int64_t rows, int64_t cols, void *stream);
int blaz_cmat_free(blaz_cmat *m, void *stream);

/* The binary64 constants of the library's DCT (Sec. III, Eq. eqdct):
 * cos_out[k*8+x] = RN(cos((2x+1) k pi / 16)), aa_out[i*8+j] = RN(alpha_i alpha_j)
 * with alpha_0 = sqrt(1/8), alpha_k = 1/2; kept_out[2t], kept_out[2t+1] =
 * (row, col) of kept code t.  Host pointers; no GPU needed. */
void blaz_constants(double cos_out[64], double aa_out[64], int32_t kept_out[56]);

/* Every stage of the compression of one 8x8 block, for inspection (Sec. II,
 * Fig. 1 pipeline and Examples 1-5).  Field by field: */
typedef struct blaz_block_stages {
    double delta[64];      /* Eq. eqnorm, row-major                                  */
    int32_t K;             /* Eq. eqslope2: number of nonzero entries of delta       */
    double sum_abs;        /* sum |delta| (the fixed pairwise tree of the specification) */
    double s;              /* Eq. eqslope: sum_abs / K (0 when K = 0)                */
    double dprime[64];     /* delta * (1/s) (0 when K = 0)                            */
    double s_max;          /* max |dprime| (prediction stage)                        */
    uint8_t psi[64];       /* Eq. eqpredict: index of the nearest of 256 reference
                              slopes s - s_max + k 2 s_max / 256, ties up; not stored
                              in the compressed block                                */
    double dct[64];        /* Eq. eqdct of dprime, all 64 coefficients               */
    double m;              /* max |dct|                                              */
    uint8_t phi;           /* Eq. eqphi                                              */
    double f;              /* the block's first element                              */
    int8_t code[BLAZ_NKEEP]; /* the 28 kept codes                                    */
} blaz_block_stages;

/* The stages above for one block, computed on the GPU on `stream` in the
 * binary64 operation order of blaz_compress (so f, s, phi and code equal the
 * compressed block's).  M: device, 64 binary64 values (row-major 8x8); out:
 * device, one blaz_block_stages.  BLAZ_ERR_NULL for a NULL pointer. */
int blaz_debug_block_stages(const double *M, blaz_block_stages *out, void *stream);

/* Compression, Sec. II (Fig. 1 pipeline; Eqs. eqnorm, eqslope, eqdct, eqphi):
 * A: device, rows x cols binary64, row-major with leading dimension lda >= cols.
 * out: rows/cols set by the caller, arrays preallocated (device).
 * Codes, phi and s are bit-identical to the binary64 operation order
 *   D(i,j) per Eq. eqnorm, interior ((Mij - Mi-1,j) + (Mij - Mi,j-1)) * 0.5;
 *   K = #{D != 0}; S = sum |D| as a fixed pairwise tree over the row-major
 *   index p (q[k] = |D_k| + |D_k+32|, k < 32, then q[k] += q[k+h] for
 *   h = 16, 8, 4, 2, 1; S = q[0]); s = S / K (0 if K = 0);
 *   D' = D * (1/s); T[u][j] = sum_v D'[u][v] cos_jv (v ascending);
 *   U[i][j] = sum_u cos_iu T[u][j] (u ascending); X = RN(alpha_i alpha_j) * U;
 *   m = max |X|; phi = trunc(127/m) clamped to [1,255];
 *   code = trunc(X * phi) saturated to [-127,127], NaN -> 0.  */
int blaz_compress(const double *A, int64_t lda, blaz_cmat *out, void *stream);
/* (blaz_compress decides most of the DCT in fp32 under a proven error bound
 * and recomputes the blocks it cannot certify in binary64, so the result is
 * the same bits; it uses 12 bytes per block of stream-ordered scratch.) */

/* Decompression (inverse of Sec. II; Eq. eqbbb read as the exact inverse of
 * Eq. eqnorm): X = code/phi on the kept positions, 0 elsewhere;
 * D_hat = s * IDCT(X); B00 = f, B0j = B0,j-1 + D_hat0j, Bi0 = Bi-1,0 + D_hati0,
 * Bij = (Bi-1,j + Bi,j-1)/2 + D_hatij.  A: device, lda >= cols. */
int blaz_decompress(const blaz_cmat *a, double *A, int64_t lda, void *stream);

/* Addition of compressed matrices, Algorithm 1 (Sec. III, Eq. eq55), per block:
 * f = f1+f2, s = s1+s2, phi = max(1, (phi1*phi2) div (phi1+phi2)),
 * alpha_k = s_k/s, beta_k = (alpha_k/phi_k)*phi,
 * code = trunc(beta1*c1 + beta2*c2) saturated to [-127,127] (0 when s == 0).
 * a, b, out: same shape; out may alias a or b entirely. Bit-exact binary64. */
int blaz_add(const blaz_cmat *a, const blaz_cmat *b, blaz_cmat *out, void *stream);

/* Subtraction (Sec. III states it works like addition; not detailed there):
 * f = f1-f2, s = s1+s2, phi as in blaz_add, code = trunc(beta1*c1 - beta2*c2). */
int blaz_sub(const blaz_cmat *a, const blaz_cmat *b, blaz_cmat *out, void *stream);

/* Multiplication by a constant, Algorithm 2: f = f1*c, s = s1*c, phi and code
 * copied.  out may equal a (in place: only f and s are rewritten). */
int blaz_scale(const blaz_cmat *a, double c, blaz_cmat *out, void *stream);

/* ---- Tunable rate ------------------------------------------------------------
 * Sec. VI names a tunable compression rate as future work (more or less
 * compression "by skewing the quantization").  These entry points keep the
 * first r rows and the first r columns of each block's DCT, r = 1..8:
 * keep(r) = 8r + (8-r)r codes per block (15, 28, 39, 48, 55, 60, 63, 64),
 * in the order rows 0..r-1 (columns 0..7), then (i, 0..r-1) for i = r..7.
 * r = 2 is the 28-code format of the functions above.  Everything else is
 * unchanged: f, s and phi (from the maximum over all 64 coefficients, so phi
 * does not depend on r), the truncated codes, Algorithms 1 and 2.  A block
 * takes 17 + keep(r) bytes: compression ratio 512 / (17 + keep(r)).
 *
 * A rate-r matrix uses the blaz_cmat descriptor with code holding
 * nb x keep(r) bytes (row-major [nb][keep(r)]); the rate is not stored in the
 * descriptor and every call names it; a code array shorter than
 * nb x keep(r) bytes is the caller's error (not detectable here).  The file
 * functions, the padded-shape variants, the batch planner and the server
 * take the 28-code format only.  r outside 1..8: BLAZ_ERR_ARG.  Results:
 * compress, add, sub and scale bit-exact with the binary64 operation order
 * above (the kernels reuse the 28-code format's certified fp32 decisions
 * with exact binary64 fix-ups, and its tensor-core decoding); decompression,
 * dots and products within that format's tolerances. */

/* keep(r), or -1 when r is outside 1..8.  No GPU needed. */
int blaz_keep_count(int r);
/* blaz_cmat_alloc with nb x keep(r) code bytes. */
int blaz_cmat_alloc_rate(blaz_cmat *m, int64_t rows, int64_t cols, int r, void *stream);
/* Compression at rate r (A: device, lda >= cols). */
int blaz_compress_rate(const double *A, int64_t lda, int r, blaz_cmat *out, void *stream);
/* Decompression at rate r: the definition of blaz_decompress with the rate's
 * kept positions.  A: device, lda >= cols.  Within 1e-12 of the block scale of
 * the exact result. */
int blaz_decompress_rate(const blaz_cmat *a, int r, double *A, int64_t lda, void *stream);
/* Algorithm 1 / its subtraction / Algorithm 2 on rate-r matrices; operands of
 * the same shape and rate; out may alias a or b. */
int blaz_add_rate(const blaz_cmat *a, const blaz_cmat *b, int r, blaz_cmat *out, void *stream);
int blaz_sub_rate(const blaz_cmat *a, const blaz_cmat *b, int r, blaz_cmat *out, void *stream);
int blaz_scale_rate(const blaz_cmat *a, double c, int r, blaz_cmat *out, void *stream);
/* Flattened dot <vec A_hat, vec B_hat> of two rate-r matrices of the same
 * shape (blaz_dot's definition; result: device, one binary64; within
 * 1e-12 sum |A_hat B_hat|; deterministic; stream-ordered scratch). */
int blaz_dot_rate(const blaz_cmat *a, const blaz_cmat *b, int r, double *result, void *stream);
/* Algorithm 3 at rate r: line i of A_hat times column j of B_hat
 * (a->cols == b->rows; 0 <= i < a->rows, 0 <= j < b->cols, else
 * BLAZ_ERR_RANGE); result: device, one binary64. */
int blaz_dot_rowcol_rate(const blaz_cmat *a, const blaz_cmat *b, int r, int64_t i, int64_t j, double *result,
                         void *stream);
/* blaz_matmul and blaz_matmul_cc with rate-r operands (same modes, layouts
 * and accuracy; the operands are decoded by the rate-r decompressor). */
int blaz_matmul_rate(const blaz_cmat *a, int r, const double *B, int64_t ldb, int64_t m, double *C, int64_t ldc,
                     int mode, void *stream);
int blaz_matmul_cc_rate(const blaz_cmat *a, const blaz_cmat *b, int r, double *C, int64_t ldc, int mode,
                        void *stream);

/* Flattened dot product <vec A_hat, vec B_hat> = sum_ij A_hat_ij B_hat_ij of
 * two compressed matrices of the same shape (A_hat, B_hat the decompressed
 * matrices).  result: device, one binary64, written in stream order.
 * Deterministic: same inputs give the same bits.  Uses stream-ordered scratch
 * (cudaMallocAsync on `stream`). */
int blaz_dot(const blaz_cmat *a, const blaz_cmat *b, double *result, void *stream);

/* blaz_dot without any device allocation (the paper has no counterpart; this
 * entry point exists for callers that cannot let a library allocate device
 * memory: a framework or server that owns all of HBM through its own
 * allocator or budget, a device or driver without stream-ordered allocation,
 * or a step that must not risk an allocation failure midway).
 * Same arguments, checks, status codes, result and determinism as blaz_dot
 * (bit-identical results on the same inputs).  Its scratch is a fixed
 * 8448-byte array in the library's device memory (every GPU that loads the
 * library holds it until the process exits): 1024 per-CTA partial sums and a
 * counter.  A call needs one partial per CTA it launches, min(ceil(nb/256),
 * 6 x SM count, 1024), i.e. at most 912 on a 152-SM GB300, so every matrix
 * size fits there (the BLAZ_ERR_RANGE check before anything is enqueued
 * cannot trigger).  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current and copies the constant tables (see above); make that first call
 * before any stream capture.  All calls share
 * the one array (the counter is cleared on the stream at the start of each
 * call): calls that can overlap on the GPU -- on different streams without
 * ordering between them -- race and must not be issued.  No cudaMalloc,
 * cudaFree or allocating library routine is called. */
int blaz_dot_noalloc(const blaz_cmat *a, const blaz_cmat *b, double *result, void *stream);

/* Dot product of line i of A_hat and column j of B_hat, Algorithm 3 (Eqs.
 * eqbbb0, eqbbb) applied block-wise: sum_k A_hat[i][k] B_hat[k][j].
 * a: n x k, b: k x m; 0 <= i < n, 0 <= j < m.  result: device, one binary64.
 * Only line i of A_hat and column j of B_hat are decompressed; uses
 * stream-ordered scratch (one partial sum per CTA). */
int blaz_dot_rowcol(const blaz_cmat *a, const blaz_cmat *b, int64_t i, int64_t j, double *result,
                    void *stream);

/* Matrix product C = A_hat * B of a compressed n x k matrix by a dense
 * binary64 k x m matrix (Sec. III, "Matrix multiplication": each block is
 * decompressed once).  B: device, ldb >= m; C: device, ldc >= m.
 * mode BLAZ_MM_FP64: binary64 products on the FP64 tensor path (DMMA);
 * mode BLAZ_MM_SPLIT_BF16: A_hat and B each split into three bf16 slices; the
 * six slice products with i+j <= 4 run as one bf16 GEMM of inner dimension
 * 6kp (kp: k rounded up to a multiple of 64, the padding zero) on the
 * 5th-generation tensor cores (tcgen05, fp32 accumulation in tensor memory),
 * stored as binary64; componentwise error about 1e-6 to 1e-5 of
 * (|A_hat||B|)_ij.  A's slices are decoded straight from the codes.
 * Uses stream-ordered scratch: 8nk bytes for the decompressed operand in
 * FP64 mode; 6kp(n+m) bytes of slices in split mode. */
enum { BLAZ_MM_FP64 = 0, BLAZ_MM_SPLIT_BF16 = 1 };
int blaz_matmul(const blaz_cmat *a, const double *B, int64_t ldb, int64_t m, double *C, int64_t ldc,
                int mode, void *stream);

/* Matrix product C = A_hat * B_hat of two compressed matrices (Sec. III,
 * "Matrix multiplication": B = B1 x B2 of compressed blocks, each
 * decompressed block computed once).  a: n x k, b: k x m (a->cols must equal
 * b->rows, else BLAZ_ERR_SHAPE); C: device, n x m binary64, ldc >= m.  Both
 * operands are decompressed once into stream-ordered scratch (8nk + 8km
 * bytes; in split mode 8km bytes for B_hat, A's slices straight from its
 * codes, and 6kp(n+m) bytes of slices), then multiplied as in blaz_matmul
 * with the same modes and accuracy (relative to |A_hat||B_hat|). */
int blaz_matmul_cc(const blaz_cmat *a, const blaz_cmat *b, double *C, int64_t ldc, int mode, void *stream);

/* ---- Matrices of any shape (padding) ----------------------------------------
 * The paper states that the method works for matrices of any dimensions
 * (Sec. IV, experimental setup) without fixing the partial blocks.  Here a
 * rows x cols matrix is compressed as its extension to ceil8(rows) x
 * ceil8(cols) that repeats the last row and the last column (edge
 * replication, which keeps the boundary blocks as smooth as the data); the
 * blaz_cmat holds that block grid, and the caller keeps the logical shape
 * (BLAZ_ERR_SHAPE unless ceil8(rows) == a->rows and ceil8(cols) == a->cols).
 * add, sub and scale apply unchanged (block-wise); the calls below restrict
 * decompression, the flattened dot and the products to the logical entries. */
int blaz_compress_padded(const double *A, int64_t lda, int64_t rows, int64_t cols, blaz_cmat *out, void *stream);
/* Writes the logical rows x cols entries only (lda >= cols). */
int blaz_decompress_padded(const blaz_cmat *a, int64_t rows, int64_t cols, double *A, int64_t lda, void *stream);
/* <vec A_hat, vec B_hat> over the logical entries: full blocks in the Gram
 * form, the partial blocks of the last block row and column decompressed in
 * binary64 and summed over their logical entries. */
int blaz_dot_padded(const blaz_cmat *a, const blaz_cmat *b, int64_t rows, int64_t cols, double *result,
                    void *stream);
/* C (n x m) = A_hat (logical n x k) * B (k x m, ldb >= m): A_hat is decoded
 * with zeros outside the logical entries, B copied into a zero-padded
 * ceil8(k)-row scratch when k is not a multiple of 8. */
int blaz_matmul_padded(const blaz_cmat *a, int64_t n, int64_t k, const double *B, int64_t ldb, int64_t m, double *C,
                       int64_t ldc, int mode, void *stream);
/* C (n x m) = A_hat (logical n x k) * B_hat (logical k x m). */
int blaz_matmul_cc_padded(const blaz_cmat *a, const blaz_cmat *b, int64_t n, int64_t k, int64_t m, double *C,
                          int64_t ldc, int mode, void *stream);

/* ---- Files: save and load compressed matrices ------------------------------
 * The 360-bit payload of Sec. II per block, stored as a little-endian file:
 *   bytes  0..7   magic "BLAZCMAT"
 *          8..11  uint32 version (1)      12..15 uint32 header size (64)
 *         16..23  int64 rows              24..31 int64 cols
 *         32..39  int64 nb = (rows/8)(cols/8)
 *         40..47  uint64 payload bytes = 45 nb
 *         48..55  uint64 FNV-1a 64-bit hash of the payload taken over
 *                 little-endian 64-bit words (last word zero-padded)
 *         56..63  zero
 *   payload: f[nb] (binary64), s[nb] (binary64), phi[nb] (uint8),
 *            code[nb][28] (int8), in block order.
 * These calls are host-side and blocking: save waits for `stream` to finish
 * the device-to-host copies, load waits for its host-to-device copies.  A
 * file is written to `path`.tmp and renamed, so a reader never sees half a
 * file.  BLAZ_ERR_IO for a failed open/read/write, BLAZ_ERR_FORMAT for a bad
 * magic, version, size or hash (checked before any device copy). */
int blaz_cmat_save(const blaz_cmat *a, const char *path, void *stream);
/* Shape stored in a file (host only; no device access). */
int blaz_cmat_file_info(const char *path, int64_t *rows, int64_t *cols);
/* Fills `out`, allocated by the caller with the file's rows and cols
 * (BLAZ_ERR_SHAPE otherwise). */
int blaz_cmat_load(const char *path, blaz_cmat *out, void *stream);

/* ---- Host buffers ----------------------------------------------------------
 * blaz_compress of a matrix in HOST memory (A: host pointer, lda >= cols;
 * page-locked memory runs at the link rate).  The matrix moves in slabs of
 * block rows (~128 MB) into a ring of device staging buffers (up to 512 MB) on a copy
 * stream owned by the library (one per device; transfers of successive calls
 * run in issue order), and `stream` compresses every slab as it lands, so
 * the compression hides behind the transfer.  Asynchronous: A must stay valid
 * and unchanged until `stream` has passed the call.  Same bits as
 * blaz_compress.  Device memory: the ring (allocated by the first call on a
 * device, grown when a call needs larger slabs, kept for later calls until
 * the process exits, so that no call waits on the host for an allocation)
 * plus 12 bytes per block of a slab, stream-ordered.  Calls on one device
 * issue their copies one call at a time. */
int blaz_compress_host(const double *A, int64_t lda, blaz_cmat *out, void *stream);
/* The packed payload of a compressed matrix (the file payload layout:
 * f[nb], s[nb], phi[nb], code[nb][28]; 45 nb bytes) to / from host memory,
 * stream-ordered (asynchronous for page-locked host memory). */
int blaz_cmat_download(const blaz_cmat *a, void *host, void *stream);
int blaz_cmat_upload(const void *host, blaz_cmat *a, void *stream);

/* ---- Batched mixed operations: one persistent, graph-captured launch ----------
 * Many compressed-matrix operations of different kinds and sizes (the
 * block-wise algorithms of Sec. III applied to whole matrices) run as one
 * persistent kernel: the plan cuts every operation into work items (a range
 * of 8x8 blocks, or a 64x64 tile of a matrix product), the CTAs take items
 * from a device-side queue in order, and the launch is captured once in a
 * CUDA graph and replayed by blaz_batch_run.  Results are the same as the
 * single-operation entry points: bit-identical for compress / add / sub /
 * scale, within the dot and product tolerances otherwise (the dot sums
 * item partials in item order, deterministically). */
enum {
    BLAZ_OP_COMPRESS = 0,   /* out = compress(A)             uses A, lda, out        */
    BLAZ_OP_DECOMPRESS = 1, /* C = decompress(a)             uses a, C, ldc          */
    BLAZ_OP_ADD = 2,        /* out = a + b (Algorithm 1)     uses a, b, out          */
    BLAZ_OP_SUB = 3,        /* out = a - b                   uses a, b, out          */
    BLAZ_OP_SCALE = 4,      /* out = c * a (Algorithm 2)     uses a, c, out          */
    BLAZ_OP_DOT = 5,        /* *result = <vec a, vec b>      uses a, b, result       */
    BLAZ_OP_MATMUL = 6      /* C = a_hat * B (binary64 DMMA) uses a, B, ldb, m, C, ldc */
};

typedef struct blaz_op {
    int32_t kind;           /* BLAZ_OP_*                                              */
    blaz_cmat a, b, out;    /* compressed operands and result (descriptors copied)   */
    const double *A;        /* COMPRESS: dense input (device), leading dimension lda */
    int64_t lda;
    double c;               /* SCALE: the constant                                    */
    double *result;         /* DOT: one binary64 (device)                             */
    const double *B;        /* MATMUL: dense k x m right operand (device), ldb        */
    int64_t ldb, m;
    double *C;              /* MATMUL / DECOMPRESS: dense output (device), ldc        */
    int64_t ldc;
} blaz_op;

typedef struct blaz_batch_cfg {
    int32_t blocks_per_item;  /* 8x8 blocks per work item (0: default 256)              */
    int32_t ctas_per_sm;      /* persistent CTAs per SM (0: default 2)                  */
    int32_t autotune;         /* 1: time candidate (blocks_per_item, ctas_per_sm) pairs
                                 on this batch and keep the fastest; the batch is then
                                 run several times, so no output may alias an input   */
} blaz_batch_cfg;

typedef struct blaz_batch_info {
    int64_t ops, items, gemm_tiles;
    int32_t blocks_per_item, ctas_per_sm, grid;
    int64_t scratch_bytes;      /* device memory owned by the plan                        */
    double tuned_ms;            /* autotune: time of the chosen configuration (else 0)    */
} blaz_batch_info;

typedef struct blaz_plan blaz_plan;

/* Validate `ops` (host array, copied), build the work list, allocate the
 * plan's device memory (descriptors, counters, partial sums, decompressed
 * operands of the products) and capture the launch in a CUDA graph.  Work is
 * enqueued on `stream` only when autotuning.  Errors: as the single-op entry
 * points, plus BLAZ_ERR_ARG for an unknown kind or an aliased output with
 * autotune. */
int blaz_batch_plan(const blaz_op *ops, int64_t nops, const blaz_batch_cfg *cfg, blaz_plan **plan, void *stream);
/* Replay the captured launch on `stream`. */
int blaz_batch_run(blaz_plan *plan, void *stream);
int blaz_batch_info_get(const blaz_plan *plan, blaz_batch_info *info);
/* Release the plan (synchronizes the device first). */
int blaz_batch_free(blaz_plan *plan);

/* ---- Request server: resident compressed matrices, continuous batching ------
 * A server owns a set of resident compressed matrices (handles) on the current
 * device and a scheduler thread.  Requests are submitted from any host
 * thread; the scheduler admits them in arrival order while the device-memory
 * budget allows (a request that does not fit waits until memory is released
 * by completing work; one that can never fit is rejected), gathers the
 * admitted requests whose operands are ready into one persistent batch launch
 * (the batch kernel above), and keeps up to `streams` such launches in flight
 * on separate streams, so requests arriving while others run are admitted as
 * slots and memory free up and their work overlaps on the device.  Every
 * result equals the single-operation entry points' result (same kernels). */
enum { BLAZ_REQ_RELEASE = 7 };  /* request kinds: BLAZ_OP_* above, plus RELEASE */
/* Request flag: every host buffer of the request is page-locked (pinned) and
 * stays valid and unmodified until the request completes; the server then
 * copies straight between it and the device instead of staging a copy. */
enum { BLAZ_REQ_PINNED = 1 };

typedef struct blaz_server_cfg {
    int64_t budget_bytes;   /* device bytes for resident matrices + in-flight work  */
    int32_t streams;        /* launches in flight at once (0: 4)                     */
    int32_t max_batch;      /* requests per launch (0: 512; 1 = one per launch)      */
    int32_t max_wait_us;    /* longest a ready request waits for company (0: 100)   */
    int32_t queue_capacity; /* submitted-but-unadmitted requests (0: 65536)          */
    int32_t matmul_mode;    /* BLAZ_MM_FP64 (DMMA inside the batch launch) or
                               BLAZ_MM_SPLIT_BF16 (tcgen05 launch after the batch)   */
} blaz_server_cfg;

typedef struct blaz_request {
    int32_t kind;           /* BLAZ_OP_COMPRESS .. BLAZ_OP_MATMUL, BLAZ_REQ_RELEASE  */
    int64_t rows, cols;     /* COMPRESS: shape of host_A                             */
    const double *host_A;   /* COMPRESS: host input, leading dimension lda (copied
                               during blaz_server_submit)                          */
    int64_t lda;
    uint64_t a, b;          /* operand handles (ADD/SUB/DOT: a, b; others: a)       */
    double c;               /* SCALE                                                 */
    const double *host_B;   /* MATMUL: host right operand, a.cols x m, ldb (copied)  */
    int64_t ldb, m;
    double *host_out;       /* DECOMPRESS: rows x cols, MATMUL: rows x m, leading
                               dimension ldo; DOT: one double.  Written by the
                               server before the request reports completion; must
                               stay valid until then.                             */
    int64_t ldo;
    int32_t flags;          /* BLAZ_REQ_PINNED or 0                                  */
} blaz_request;

typedef struct blaz_result {
    int32_t status;         /* BLAZ_OK, 1 = still pending, or a BLAZ_ERR_* code      */
    uint64_t handle;        /* COMPRESS/ADD/SUB/SCALE: the new resident matrix       */
    double value;           /* DOT                                                   */
    double latency_us;      /* submission to completion                              */
} blaz_result;

typedef struct blaz_server_stats {
    int64_t submitted, completed, rejected, launches, resident_matrices, resident_bytes, peak_bytes;
    double p50_us, p99_us, mean_batch, throughput_rps;
} blaz_server_stats;

typedef struct blaz_server blaz_server;

int blaz_server_create(const blaz_server_cfg *cfg, blaz_server **srv);
/* Validates and enqueues; returns a ticket.  BLAZ_ERR_BUSY when the queue is
 * full (retry later), BLAZ_ERR_BUDGET when the request alone exceeds the
 * budget, BLAZ_ERR_SHAPE / NULL / LD / ARG for invalid requests. */
int blaz_server_submit(blaz_server *srv, const blaz_request *req, uint64_t *ticket);
/* Non-blocking: status 1 while pending.  A completed ticket is forgotten after
 * it is reported once. */
int blaz_server_poll(blaz_server *srv, uint64_t ticket, blaz_result *res);
/* Blocks until the ticket completes or timeout_us passes (BLAZ_ERR_TIMEOUT). */
int blaz_server_wait(blaz_server *srv, uint64_t ticket, blaz_result *res, int64_t timeout_us);
/* Device descriptor of a resident matrix (read-only view, valid until released). */
int blaz_server_cmat(blaz_server *srv, uint64_t handle, blaz_cmat *out);
int blaz_server_stats_get(blaz_server *srv, blaz_server_stats *st);
/* Drains in-flight work, frees every resident matrix, stops the scheduler. */
int blaz_server_destroy(blaz_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* BLAZ_H */
