/*
 * blaz_oracle.c -- plain, slow, single-threaded CPU oracle of the blaz
 * compressed-matrix method (Martel, "Compressed Matrix Computations",
 * arXiv 2202.13007).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Build: cc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (no FMA contraction, so every binary64 operation below is one IEEE-754
 * round-to-nearest-even operation, in the order written).
 *
 * The binary64 operation order written here is the arithmetic specification
 * that the GPU compressor, add and scale reproduce bit for bit:
 *
 *   compress (Sec. II, Eqs. eqnorm, eqslope, eqphi):
 *     f = M00
 *     D(i,j) per Eq. eqnorm; the interior case is ((Mij-Mi-1j)+(Mij-Mij-1))*0.5
 *     K = #{D != 0}; S = sum |D| as a fixed pairwise tree over the row-major
 *     index (|D_k| + |D_k+32| for k < 32, then strides 16, 8, 4, 2, 1);
 *     s = S / K (s = 0 when K = 0: constant block)
 *     r = 1 / s ; D'(i,j) = D(i,j) * r           (D' = (1/s) D literally)
 *     DCT-II, Eq. eqdct with alpha_i alpha_j outside the double sum:
 *       COS[k][x] = RN(cos((2x+1) k pi / 16)),  AA[i][j] = RN(alpha_i alpha_j)
 *       T[u][j] = sum_v D'[u][v]*COS[j][v]  (inner sum, v = 0..7, left to right)
 *       U[i][j] = sum_u COS[i][u]*T[u][j]   (outer sum, u = 0..7, left to right)
 *       X[i][j] = AA[i][j] * U[i][j]
 *     m = max |X| over all 64 coefficients
 *     phi = trunc(127 / m) clamped to [1, 255]   (127/0 = inf -> 255)
 *     C = trunc(X * phi) on the first two rows and columns, saturated to
 *         [-127, 127]; NaN -> 0.  Kept order: row 0 (j=0..7), row 1 (j=0..7),
 *         then (i,0),(i,1) for i = 2..7.
 *   add (Algorithm 1), scale (Algorithm 2): literal, see the functions.
 *
 * Decompression, dot products and matrix multiplication are floating-point
 * results compared within a tolerance; they are written here as the plain
 * definitions (inverse DCT of C/phi with the 36 dropped coefficients set to
 * zero, times s, followed by the exact inverse of Eq. eqnorm).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BLK 8
#define NKEEP 28

/* Status codes returned by the matrix-level functions. */
#define ORC_OK 0
#define ORC_ERR_SHAPE (-1)
#define ORC_ERR_NULL (-2)
#define ORC_ERR_LD (-3)
#define ORC_ERR_RANGE (-4)

/* ------------------------------------------------------------------------ */
/* DCT-II constants (Sec. III, Eq. eqdct): COS[k][x] = RN(cos((2x+1)k pi/16)) */
/* and AA[i][j] = RN(alpha_i alpha_j), alpha_0 = sqrt(1/8), alpha_k = 1/2.    */
/* Evaluated in long double and rounded once to binary64.  The tests pin both */
/* tables against a 50-digit evaluation.                                      */
/* ------------------------------------------------------------------------ */
static double COS[BLK][BLK];
static double AA[BLK][BLK];
static int cm_ready = 0;

static void cm_init(void)
{
    if (cm_ready) return;
    const long double pi = 3.14159265358979323846264338327950288L;
    long double alpha[BLK];
    for (int k = 0; k < BLK; ++k) alpha[k] = (k == 0) ? sqrtl(1.0L / 8.0L) : 0.5L;
    for (int k = 0; k < BLK; ++k)
        for (int x = 0; x < BLK; ++x) {
            long double ang = (long double)((2 * x + 1) * k) * pi / 16.0L;
            COS[k][x] = (double)cosl(ang);
        }
    for (int i = 0; i < BLK; ++i)
        for (int j = 0; j < BLK; ++j) AA[i][j] = (double)(alpha[i] * alpha[j]);
    cm_ready = 1;
}

void blazo_dct_tables(double cos_out[64], double aa_out[64])
{
    cm_init();
    for (int k = 0; k < BLK; ++k)
        for (int x = 0; x < BLK; ++x) {
            cos_out[k * BLK + x] = COS[k][x];
            aa_out[k * BLK + x] = AA[k][x];
        }
}

/* Position (row, col) of kept code number t, t = 0..27 (first two rows, then
 * the first two columns of rows 2..7). */
static void kept_pos(int t, int *i, int *j)
{
    if (t < 16) { *i = t / 8; *j = t % 8; }
    else { int q = t - 16; *i = 2 + q / 2; *j = q % 2; }
}

void blazo_kept_positions(int32_t out[56])
{
    for (int t = 0; t < NKEEP; ++t) kept_pos(t, &out[2 * t], &out[2 * t + 1]);
}

static int8_t quantize_code(double v)
{
    if (v != v) return 0;
    if (v >= 127.0) return 127;
    if (v <= -127.0) return -127;
    return (int8_t)(int)v;            /* C conversion truncates toward zero */
}

/* All intermediate stages of compressing one block (Sec. II, Ex. 1-5).       */
typedef struct {
    double delta[64];      /* Eq. eqnorm                                  */
    int32_t K;             /* Eq. eqslope2: number of nonzero deltas      */
    double sum_abs;        /* sum |delta|, fixed pairwise tree            */
    double s;              /* Eq. eqslope                                 */
    double dprime[64];     /* (1/s) * delta                               */
    double s_max;          /* max |dprime| (prediction stage)             */
    uint8_t psi[64];       /* Eq. eqpredict (not part of the payload)     */
    double dct[64];        /* Eq. eqdct applied to dprime                 */
    double m;              /* max |dct|                                   */
    uint8_t phi;           /* Eq. eqphi, truncated to an 8-bit integer    */
    double f;              /* M00                                         */
    int8_t code[NKEEP];    /* kept, re-scaled, truncated coefficients     */
} blazo_stages;

void blazo_block_stages(const double *M, blazo_stages *st)
{
    cm_init();
    memset(st, 0, sizeof(*st));
    st->f = M[0];

    /* Eq. eqnorm */
    double *d = st->delta;
    for (int i = 0; i < BLK; ++i) {
        for (int j = 0; j < BLK; ++j) {
            double v;
            if (i == 0 && j == 0) v = 0.0;
            else if (i == 0) v = M[j] - M[j - 1];
            else if (j == 0) v = M[i * BLK] - M[(i - 1) * BLK];
            else {
                double a = M[i * BLK + j] - M[(i - 1) * BLK + j];
                double b = M[i * BLK + j] - M[i * BLK + j - 1];
                v = (a + b) * 0.5;
            }
            d[i * BLK + j] = v;
        }
    }

    /* Eqs. eqslope, eqslope2.  The paper leaves the order of the sum open;
     * it is a fixed pairwise tree over the row-major index p: first
     * tree[k] = |d[k]| + |d[k+32]| for k < 32, then tree[k] += tree[k+h]
     * for h = 16, 8, 4, 2, 1 (k < h); S = tree[0]. */
    int K = 0;
    for (int p = 0; p < 64; ++p)
        if (d[p] != 0.0) ++K;
    double tree[32];
    for (int k = 0; k < 32; ++k) tree[k] = fabs(d[k]) + fabs(d[k + 32]);
    for (int h = 16; h >= 1; h /= 2)
        for (int k = 0; k < h; ++k) tree[k] = tree[k] + tree[k + h];
    double S = tree[0];
    st->K = K;
    st->sum_abs = S;
    double s = 0.0;
    if (K > 0) {
        s = S / (double)K;
        double r = 1.0 / s;
        for (int p = 0; p < 64; ++p) st->dprime[p] = d[p] * r;
    }
    st->s = s;

    /* Prediction, Eq. eqpredict: 256 equidistant reference slopes on
     * [s - s_max, s + s_max], index of the nearest one (ties away from the
     * lower slope).  Kept for inspection; it does not enter the payload. */
    double smax = 0.0;
    for (int p = 0; p < 64; ++p) {
        double a = fabs(st->dprime[p]);
        if (a > smax) smax = a;
    }
    st->s_max = smax;
    if (smax > 0.0) {
        double lo = s - smax;
        double step = (2.0 * smax) / 256.0;
        for (int p = 0; p < 64; ++p) {
            double k = floor((st->dprime[p] - lo) / step + 0.5);
            if (k < 0.0) k = 0.0;
            if (k > 255.0) k = 255.0;
            st->psi[p] = (uint8_t)k;
        }
    }

    /* Eq. eqdct: DCT-II of dprime; the double sum is evaluated as an inner
     * sum over v and an outer sum over u, and alpha_i alpha_j multiplies the
     * result as in the equation. */
    double T[BLK][BLK];
    for (int u = 0; u < BLK; ++u) {
        for (int j = 0; j < BLK; ++j) {
            double acc = st->dprime[u * BLK + 0] * COS[j][0];
            for (int v = 1; v < BLK; ++v) acc = acc + st->dprime[u * BLK + v] * COS[j][v];
            T[u][j] = acc;
        }
    }
    for (int i = 0; i < BLK; ++i) {
        for (int j = 0; j < BLK; ++j) {
            double acc = COS[i][0] * T[0][j];
            for (int u = 1; u < BLK; ++u) acc = acc + COS[i][u] * T[u][j];
            st->dct[i * BLK + j] = AA[i][j] * acc;
        }
    }

    /* Eq. eqphi */
    double m = 0.0;
    for (int p = 0; p < 64; ++p) {
        double a = fabs(st->dct[p]);
        if (a > m) m = a;
    }
    st->m = m;
    double q = 127.0 / m;
    int phi;
    if (!(q < 255.0)) phi = 255;
    else {
        phi = (int)q;
        if (phi < 1) phi = 1;
    }
    st->phi = (uint8_t)phi;
    double phid = (double)phi;

    for (int t = 0; t < NKEEP; ++t) {
        int i, j;
        kept_pos(t, &i, &j);
        st->code[t] = quantize_code(st->dct[i * BLK + j] * phid);
    }
}

void blazo_compress_block(const double *M, double *f, double *s, uint8_t *phi, int8_t *code)
{
    blazo_stages st;
    blazo_block_stages(M, &st);
    *f = st.f;
    *s = st.s;
    *phi = st.phi;
    memcpy(code, st.code, NKEEP);
}

/* Decompression of one block: X = C/phi on the kept positions and zero
 * elsewhere; P = inverse DCT of X; delta_hat = s * P; then the exact inverse
 * of Eq. eqnorm (Eq. eqbbb with P read at (0,j), (i,0) and (i,j)). */
void blazo_decompress_block(double f, double s, uint8_t phi, const int8_t *code, double *M)
{
    cm_init();
    double X[BLK][BLK];
    memset(X, 0, sizeof(X));
    for (int t = 0; t < NKEEP; ++t) {
        int i, j;
        kept_pos(t, &i, &j);
        X[i][j] = (double)code[t] / (double)phi;
    }
    /* inverse DCT-II (the transpose of the orthonormal DCT-II):
     * P[u][v] = sum_i sum_j alpha_i alpha_j X[i][j] cos_iu cos_jv */
    double Y[BLK][BLK];
    for (int i = 0; i < BLK; ++i)
        for (int j = 0; j < BLK; ++j) Y[i][j] = AA[i][j] * X[i][j];
    double Q[BLK][BLK];
    for (int i = 0; i < BLK; ++i)
        for (int v = 0; v < BLK; ++v) {
            double acc = Y[i][0] * COS[0][v];
            for (int j = 1; j < BLK; ++j) acc = acc + Y[i][j] * COS[j][v];
            Q[i][v] = acc;
        }
    double P[BLK][BLK];
    for (int u = 0; u < BLK; ++u)
        for (int v = 0; v < BLK; ++v) {
            double acc = COS[0][u] * Q[0][v];
            for (int i = 1; i < BLK; ++i) acc = acc + COS[i][u] * Q[i][v];
            P[u][v] = acc;
        }
    for (int i = 0; i < BLK; ++i)
        for (int j = 0; j < BLK; ++j) {
            double dh = s * P[i][j];
            double v;
            if (i == 0 && j == 0) v = f;
            else if (i == 0) v = M[j - 1] + dh;
            else if (j == 0) v = M[(i - 1) * BLK] + dh;
            else v = (M[(i - 1) * BLK + j] + M[i * BLK + j - 1]) * 0.5 + dh;
            M[i * BLK + j] = v;
        }
}

/* Algorithm 1: addition of two compressed blocks.  With sub != 0 the same
 * algorithm subtracts (Sec. III: subtraction works like addition): the first
 * elements are subtracted, the slopes still add (s = s1 + s2 keeps the
 * combined block's scale positive) and the rescaled codes are subtracted. */
static void addsub_block_n(int sub, int ncodes, double f1, double s1, uint8_t phi1, const int8_t *c1,
                           double f2, double s2, uint8_t phi2, const int8_t *c2,
                           double *f, double *s, uint8_t *phi, int8_t *c)
{
    double fs = sub ? f1 - f2 : f1 + f2;
    double ss = s1 + s2;
    int p1 = phi1, p2 = phi2;
    int ph = (p1 * p2) / (p1 + p2);         /* integer product and quotient */
    if (ph < 1) ph = 1;
    *f = fs;
    *s = ss;
    *phi = (uint8_t)ph;
    if (ss == 0.0) {
        memset(c, 0, (size_t)ncodes);
        return;
    }
    double a1 = s1 / ss;
    double a2 = s2 / ss;
    double b1 = (a1 / (double)p1) * (double)ph;
    double b2 = (a2 / (double)p2) * (double)ph;
    for (int t = 0; t < ncodes; ++t)
        c[t] = quantize_code(sub ? b1 * (double)c1[t] - b2 * (double)c2[t]
                                 : b1 * (double)c1[t] + b2 * (double)c2[t]);
}

static void addsub_block(int sub, double f1, double s1, uint8_t phi1, const int8_t *c1,
                         double f2, double s2, uint8_t phi2, const int8_t *c2,
                         double *f, double *s, uint8_t *phi, int8_t *c)
{
    addsub_block_n(sub, NKEEP, f1, s1, phi1, c1, f2, s2, phi2, c2, f, s, phi, c);
}

void blazo_add_block(double f1, double s1, uint8_t phi1, const int8_t *c1,
                     double f2, double s2, uint8_t phi2, const int8_t *c2,
                     double *f, double *s, uint8_t *phi, int8_t *c)
{
    addsub_block(0, f1, s1, phi1, c1, f2, s2, phi2, c2, f, s, phi, c);
}

void blazo_sub_block(double f1, double s1, uint8_t phi1, const int8_t *c1,
                     double f2, double s2, uint8_t phi2, const int8_t *c2,
                     double *f, double *s, uint8_t *phi, int8_t *c)
{
    addsub_block(1, f1, s1, phi1, c1, f2, s2, phi2, c2, f, s, phi, c);
}

/* Algorithm 2: multiplication of a compressed block by a constant. */
void blazo_scale_block(double f1, double s1, uint8_t phi1, const int8_t *c1, double cst,
                       double *f, double *s, uint8_t *phi, int8_t *c)
{
    *f = f1 * cst;
    *s = s1 * cst;
    *phi = phi1;
    memcpy(c, c1, NKEEP);
}

/* ------------------------------------------------------------------------ */
/* Matrix level: blocks in row-major order over the (rows/8) x (cols/8)     */
/* block grid; structure of arrays f[nb], s[nb], phi[nb], code[nb][28].      */
/* ------------------------------------------------------------------------ */
static int check_shape(int64_t rows, int64_t cols)
{
    if (rows < 0 || cols < 0 || rows % BLK || cols % BLK) return ORC_ERR_SHAPE;
    return ORC_OK;
}

int blazo_compress(const double *A, int64_t rows, int64_t cols, int64_t lda,
                   double *f, double *s, uint8_t *phi, int8_t *code)
{
    int e = check_shape(rows, cols);
    if (e) return e;
    if (lda < cols) return ORC_ERR_LD;
    int64_t nbc = cols / BLK;
    double M[64];
    for (int64_t bi = 0; bi < rows / BLK; ++bi)
        for (int64_t bj = 0; bj < nbc; ++bj) {
            for (int i = 0; i < BLK; ++i)
                for (int j = 0; j < BLK; ++j)
                    M[i * BLK + j] = A[(bi * BLK + i) * lda + bj * BLK + j];
            int64_t b = bi * nbc + bj;
            blazo_compress_block(M, &f[b], &s[b], &phi[b], &code[b * NKEEP]);
        }
    return ORC_OK;
}

/* Compress only the listed blocks (block indices into the block grid); used to
 * check sampled blocks of very large matrices. */
int blazo_compress_blocks(const double *A, int64_t rows, int64_t cols, int64_t lda,
                          const int64_t *blocks, int64_t nsel,
                          double *f, double *s, uint8_t *phi, int8_t *code)
{
    int e = check_shape(rows, cols);
    if (e) return e;
    if (lda < cols) return ORC_ERR_LD;
    int64_t nbc = cols / BLK, nb = (rows / BLK) * nbc;
    double M[64];
    for (int64_t q = 0; q < nsel; ++q) {
        int64_t b = blocks[q];
        if (b < 0 || b >= nb) return ORC_ERR_RANGE;
        int64_t bi = b / nbc, bj = b % nbc;
        for (int i = 0; i < BLK; ++i)
            for (int j = 0; j < BLK; ++j)
                M[i * BLK + j] = A[(bi * BLK + i) * lda + bj * BLK + j];
        blazo_compress_block(M, &f[q], &s[q], &phi[q], &code[q * NKEEP]);
    }
    return ORC_OK;
}

int blazo_decompress(const double *f, const double *s, const uint8_t *phi, const int8_t *code,
                     int64_t rows, int64_t cols, double *A, int64_t lda)
{
    int e = check_shape(rows, cols);
    if (e) return e;
    if (lda < cols) return ORC_ERR_LD;
    int64_t nbc = cols / BLK;
    double M[64];
    for (int64_t bi = 0; bi < rows / BLK; ++bi)
        for (int64_t bj = 0; bj < nbc; ++bj) {
            int64_t b = bi * nbc + bj;
            blazo_decompress_block(f[b], s[b], phi[b], &code[b * NKEEP], M);
            for (int i = 0; i < BLK; ++i)
                for (int j = 0; j < BLK; ++j)
                    A[(bi * BLK + i) * lda + bj * BLK + j] = M[i * BLK + j];
        }
    return ORC_OK;
}

int blazo_add(int64_t nb,
              const double *f1, const double *s1, const uint8_t *phi1, const int8_t *c1,
              const double *f2, const double *s2, const uint8_t *phi2, const int8_t *c2,
              double *f, double *s, uint8_t *phi, int8_t *c)
{
    for (int64_t b = 0; b < nb; ++b)
        blazo_add_block(f1[b], s1[b], phi1[b], &c1[b * NKEEP], f2[b], s2[b], phi2[b], &c2[b * NKEEP],
                        &f[b], &s[b], &phi[b], &c[b * NKEEP]);
    return ORC_OK;
}

int blazo_sub(int64_t nb,
              const double *f1, const double *s1, const uint8_t *phi1, const int8_t *c1,
              const double *f2, const double *s2, const uint8_t *phi2, const int8_t *c2,
              double *f, double *s, uint8_t *phi, int8_t *c)
{
    for (int64_t b = 0; b < nb; ++b)
        blazo_sub_block(f1[b], s1[b], phi1[b], &c1[b * NKEEP], f2[b], s2[b], phi2[b], &c2[b * NKEEP],
                        &f[b], &s[b], &phi[b], &c[b * NKEEP]);
    return ORC_OK;
}

int blazo_scale(int64_t nb, const double *f1, const double *s1, const uint8_t *phi1,
                const int8_t *c1, double cst, double *f, double *s, uint8_t *phi, int8_t *c)
{
    for (int64_t b = 0; b < nb; ++b)
        blazo_scale_block(f1[b], s1[b], phi1[b], &c1[b * NKEEP], cst, &f[b], &s[b], &phi[b],
                          &c[b * NKEEP]);
    return ORC_OK;
}

/* Neumaier compensated summation: the plain sum with its rounding error
 * carried separately, so that the reference dot products are accurate to a
 * few units in the last place whatever their length. */
typedef struct { double sum, comp; } csum;
static void csum_add(csum *a, double x)
{
    double t = a->sum + x;
    if (fabs(a->sum) >= fabs(x)) a->comp += (a->sum - t) + x;
    else a->comp += (x - t) + a->sum;
    a->sum = t;
}

/* Flattened dot product <vec A_hat, vec B_hat> of two compressed matrices of
 * the same shape: the sum over all elements of the product of the two
 * decompressed matrices.  Also returns sum |A_hat| |B_hat| (for the error
 * bound). */
int blazo_dot(const double *fa, const double *sa, const uint8_t *pa, const int8_t *ca,
              const double *fb, const double *sb, const uint8_t *pb, const int8_t *cb,
              int64_t nb, double *result, double *abs_result)
{
    csum acc = {0.0, 0.0}, aacc = {0.0, 0.0};
    double Ma[64], Mb[64];
    for (int64_t b = 0; b < nb; ++b) {
        blazo_decompress_block(fa[b], sa[b], pa[b], &ca[b * NKEEP], Ma);
        blazo_decompress_block(fb[b], sb[b], pb[b], &cb[b * NKEEP], Mb);
        for (int p = 0; p < 64; ++p) {
            csum_add(&acc, Ma[p] * Mb[p]);
            csum_add(&aacc, fabs(Ma[p] * Mb[p]));
        }
    }
    *result = acc.sum + acc.comp;
    if (abs_result) *abs_result = aacc.sum + aacc.comp;
    return ORC_OK;
}

/* Decompress row i of a compressed rows x cols matrix into out[cols]. */
static void decompress_row(const double *f, const double *s, const uint8_t *phi,
                           const int8_t *code, int64_t cols, int64_t i, double *out)
{
    int64_t nbc = cols / BLK, bi = i / BLK;
    double M[64];
    for (int64_t bj = 0; bj < nbc; ++bj) {
        int64_t b = bi * nbc + bj;
        blazo_decompress_block(f[b], s[b], phi[b], &code[b * NKEEP], M);
        for (int j = 0; j < BLK; ++j) out[bj * BLK + j] = M[(i % BLK) * BLK + j];
    }
}

/* Decompress column j of a compressed rows x cols matrix into out[rows]. */
static void decompress_col(const double *f, const double *s, const uint8_t *phi,
                           const int8_t *code, int64_t rows, int64_t cols, int64_t j, double *out)
{
    int64_t nbc = cols / BLK, bj = j / BLK;
    double M[64];
    for (int64_t bi = 0; bi < rows / BLK; ++bi) {
        int64_t b = bi * nbc + bj;
        blazo_decompress_block(f[b], s[b], phi[b], &code[b * NKEEP], M);
        for (int i = 0; i < BLK; ++i) out[bi * BLK + i] = M[i * BLK + (j % BLK)];
    }
}

/* Algorithm 3 generalised to matrices: line i of compressed A (ra x ca)
 * times column j of compressed B (ca x cb), Eq. eqbbb0. */
int blazo_dot_rowcol(const double *fa, const double *sa, const uint8_t *pa, const int8_t *ca_,
                     int64_t ra, int64_t ca,
                     const double *fb, const double *sb, const uint8_t *pb, const int8_t *cb_,
                     int64_t cb, int64_t i, int64_t j, double *result, double *abs_result)
{
    if (check_shape(ra, ca) || check_shape(ca, cb)) return ORC_ERR_SHAPE;
    if (i < 0 || i >= ra || j < 0 || j >= cb) return ORC_ERR_RANGE;
    double *row = (double *)malloc(sizeof(double) * (size_t)(ca ? ca : 1));
    double *col = (double *)malloc(sizeof(double) * (size_t)(ca ? ca : 1));
    decompress_row(fa, sa, pa, ca_, ca, i, row);
    decompress_col(fb, sb, pb, cb_, ca, cb, j, col);
    csum r = {0.0, 0.0}, ar = {0.0, 0.0};
    for (int64_t k = 0; k < ca; ++k) {
        csum_add(&r, row[k] * col[k]);
        csum_add(&ar, fabs(row[k] * col[k]));
    }
    free(row);
    free(col);
    *result = r.sum + r.comp;
    if (abs_result) *abs_result = ar.sum + ar.comp;
    return ORC_OK;
}

/* Matrix product C = A_hat * B of a compressed n x k matrix A by a dense
 * binary64 k x m matrix B (row-major, ldb), for the listed output entries
 * (rows ii[q], cols jj[q]); also returns sum_k |A_hat[i][k]| |B[k][j]|.
 * With nsel = n*m and the identity lists this is the full product. */
int blazo_matmul_entries(const double *fa, const double *sa, const uint8_t *pa, const int8_t *ca_,
                         int64_t n, int64_t k, const double *B, int64_t ldb, int64_t m,
                         const int64_t *ii, const int64_t *jj, int64_t nsel,
                         double *out, double *abs_out)
{
    if (check_shape(n, k)) return ORC_ERR_SHAPE;
    if (ldb < m) return ORC_ERR_LD;
    double *row = (double *)malloc(sizeof(double) * (size_t)(k ? k : 1));
    int64_t cur = -1;
    for (int64_t q = 0; q < nsel; ++q) {
        int64_t i = ii[q], j = jj[q];
        if (i < 0 || i >= n || j < 0 || j >= m) { free(row); return ORC_ERR_RANGE; }
        if (i != cur) { decompress_row(fa, sa, pa, ca_, k, i, row); cur = i; }
        csum r = {0.0, 0.0}, ar = {0.0, 0.0};
        for (int64_t t = 0; t < k; ++t) {
            csum_add(&r, row[t] * B[t * ldb + j]);
            csum_add(&ar, fabs(row[t] * B[t * ldb + j]));
        }
        out[q] = r.sum + r.comp;
        if (abs_out) abs_out[q] = ar.sum + ar.comp;
    }
    free(row);
    return ORC_OK;
}

/* Full product C = A_hat * B (n x m, ldc), plain i-j-k loops. */
int blazo_matmul(const double *fa, const double *sa, const uint8_t *pa, const int8_t *ca_,
                 int64_t n, int64_t k, const double *B, int64_t ldb, int64_t m,
                 double *C, int64_t ldc)
{
    if (check_shape(n, k)) return ORC_ERR_SHAPE;
    if (ldb < m || ldc < m) return ORC_ERR_LD;
    double *Ah = (double *)malloc(sizeof(double) * (size_t)(n * k > 0 ? n * k : 1));
    int e = blazo_decompress(fa, sa, pa, ca_, n, k, Ah, k);
    if (e) { free(Ah); return e; }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < m; ++j) {
            csum r = {0.0, 0.0};
            for (int64_t t = 0; t < k; ++t) csum_add(&r, Ah[i * k + t] * B[t * ldb + j]);
            C[i * ldc + j] = r.sum + r.comp;
        }
    free(Ah);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Tunable rate.  Sec. VI names a tunable compression rate as future work     */
/* ("by skewing the quantization"); the reading taken here keeps the first r  */
/* rows and the first r columns of the DCT, r = 1..8 (r = 2 is Sec. II's      */
/* format): keep(r) = 8 r + (8 - r) r codes per block, in the order rows      */
/* 0..r-1 (j = 0..7), then (i, 0..r-1) for i = r..7.  Every other stage is    */
/* unchanged: f, s and phi (from the maximum over all 64 coefficients, so it  */
/* does not depend on r), the truncation of X phi, Algorithms 1 and 2.        */
/* ------------------------------------------------------------------------ */
static int keep_count(int r) { return 8 * r + (8 - r) * r; }

static void kept_pos_rate(int r, int t, int *i, int *j)
{
    if (t < 8 * r) { *i = t / 8; *j = t % 8; }
    else { int q = t - 8 * r; *i = r + q / r; *j = q % r; }
}

int blazo_keep_count(int r) { return (r >= 1 && r <= 8) ? keep_count(r) : -1; }

void blazo_compress_block_rate(const double *M, int r, double *f, double *s, uint8_t *phi, int8_t *code)
{
    blazo_stages st;
    blazo_block_stages(M, &st);
    *f = st.f;
    *s = st.s;
    *phi = st.phi;
    double phid = (double)st.phi;
    for (int t = 0; t < keep_count(r); ++t) {
        int i, j;
        kept_pos_rate(r, t, &i, &j);
        code[t] = quantize_code(st.dct[i * BLK + j] * phid);
    }
}

/* The same definition as blazo_decompress_block with the rate's kept set. */
void blazo_decompress_block_rate(double f, double s, uint8_t phi, const int8_t *code, int r, double *M)
{
    cm_init();
    double X[BLK][BLK];
    memset(X, 0, sizeof(X));
    for (int t = 0; t < keep_count(r); ++t) {
        int i, j;
        kept_pos_rate(r, t, &i, &j);
        X[i][j] = (double)code[t] / (double)phi;
    }
    double Y[BLK][BLK];
    for (int i = 0; i < BLK; ++i)
        for (int j = 0; j < BLK; ++j) Y[i][j] = AA[i][j] * X[i][j];
    double Q[BLK][BLK];
    for (int i = 0; i < BLK; ++i)
        for (int v = 0; v < BLK; ++v) {
            double acc = Y[i][0] * COS[0][v];
            for (int j = 1; j < BLK; ++j) acc = acc + Y[i][j] * COS[j][v];
            Q[i][v] = acc;
        }
    double P[BLK][BLK];
    for (int u = 0; u < BLK; ++u)
        for (int v = 0; v < BLK; ++v) {
            double acc = COS[0][u] * Q[0][v];
            for (int i = 1; i < BLK; ++i) acc = acc + COS[i][u] * Q[i][v];
            P[u][v] = acc;
        }
    for (int i = 0; i < BLK; ++i)
        for (int j = 0; j < BLK; ++j) {
            double dh = s * P[i][j];
            double v;
            if (i == 0 && j == 0) v = f;
            else if (i == 0) v = M[j - 1] + dh;
            else if (j == 0) v = M[(i - 1) * BLK] + dh;
            else v = (M[(i - 1) * BLK + j] + M[i * BLK + j - 1]) * 0.5 + dh;
            M[i * BLK + j] = v;
        }
}

int blazo_compress_rate(const double *A, int64_t rows, int64_t cols, int64_t lda, int r,
                        double *f, double *s, uint8_t *phi, int8_t *code)
{
    int e = check_shape(rows, cols);
    if (e) return e;
    if (lda < cols) return ORC_ERR_LD;
    if (r < 1 || r > 8) return ORC_ERR_RANGE;
    int64_t nbc = cols / BLK, nk = keep_count(r);
    double M[64];
    for (int64_t bi = 0; bi < rows / BLK; ++bi)
        for (int64_t bj = 0; bj < nbc; ++bj) {
            for (int i = 0; i < BLK; ++i)
                for (int j = 0; j < BLK; ++j)
                    M[i * BLK + j] = A[(bi * BLK + i) * lda + bj * BLK + j];
            int64_t b = bi * nbc + bj;
            blazo_compress_block_rate(M, r, &f[b], &s[b], &phi[b], &code[b * nk]);
        }
    return ORC_OK;
}

int blazo_decompress_rate(const double *f, const double *s, const uint8_t *phi, const int8_t *code, int r,
                          int64_t rows, int64_t cols, double *A, int64_t lda)
{
    int e = check_shape(rows, cols);
    if (e) return e;
    if (lda < cols) return ORC_ERR_LD;
    if (r < 1 || r > 8) return ORC_ERR_RANGE;
    int64_t nbc = cols / BLK, nk = keep_count(r);
    double M[64];
    for (int64_t bi = 0; bi < rows / BLK; ++bi)
        for (int64_t bj = 0; bj < nbc; ++bj) {
            int64_t b = bi * nbc + bj;
            blazo_decompress_block_rate(f[b], s[b], phi[b], &code[b * nk], r, M);
            for (int i = 0; i < BLK; ++i)
                for (int j = 0; j < BLK; ++j)
                    A[(bi * BLK + i) * lda + bj * BLK + j] = M[i * BLK + j];
        }
    return ORC_OK;
}

int blazo_add_rate(int64_t nb, int r, int sub,
                   const double *f1, const double *s1, const uint8_t *phi1, const int8_t *c1,
                   const double *f2, const double *s2, const uint8_t *phi2, const int8_t *c2,
                   double *f, double *s, uint8_t *phi, int8_t *c)
{
    if (r < 1 || r > 8) return ORC_ERR_RANGE;
    int nk = keep_count(r);
    for (int64_t b = 0; b < nb; ++b)
        addsub_block_n(sub, nk, f1[b], s1[b], phi1[b], &c1[b * nk], f2[b], s2[b], phi2[b], &c2[b * nk],
                       &f[b], &s[b], &phi[b], &c[b * nk]);
    return ORC_OK;
}
