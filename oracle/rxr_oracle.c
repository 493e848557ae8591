/*
 * rxr_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the
 * randomized XR-preconditioned CholeskyQR of Fan, Guo & Lin ("A Novel
 * Randomized XR-Based Preconditioned CholeskyQR Algorithm").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA implementation and must never be used as a fallback for it.
 *
 * Every routine follows a passage of the paper or a textbook definition and is
 * written for a reader to check by eye: no blocking, fusion or reordering beyond
 * what the definition states.  Matrices are column-major (LAPACK style): entry
 * (i, j) of an m x n matrix with leading dimension ld is p[i + j*ld].
 *
 * Compile with -ffp-contract=off: the FP32 normal generator must round exactly
 * as written (no fused multiply-adds other than the explicit fmaf calls).
 *
 * Built with -fopenmp (the multi-core CPU baseline), the loops over
 * independent 256-row blocks and over independent rows run on all host cores.
 * Each block's partial sum and each row's result is computed exactly as in the
 * serial build, and the partial sums are combined in the same order, so both
 * builds return the same bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads the parallel loops use: 1 in the serial build. */
int rxo_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Status codes (same meaning as the library's, defined here independently). */
#define RXO_OK 0
#define RXO_SKETCH_SINGULAR 1
#define RXO_CHOL_BREAKDOWN 2
#define RXO_NONFINITE 3

#define RXO_VARIANT_LU 0
#define RXO_VARIANT_QR 1
#define RXO_VARIANT_NONE 2 /* no preconditioner: plain CholeskyQR repeated (Alg. 1/2) */
#define RXO_SKETCH_ROWS 16 /* flag: row extraction (Section 2.3) instead of the Gaussian sketch */

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  One round maps the */
/* counter (c0,c1,c2,c3) with key (k0,k1) to                                  */
/*   (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0));               */
/* the key is advanced by the Weyl constants between rounds; ten rounds.      */
/* ------------------------------------------------------------------------- */
void rxo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* FP32 natural logarithm on (0, 1], written from the mathematics:            */
/*   u = 2^e * x with x in [sqrt(1/2), sqrt(2)];                              */
/*   log x = 2 atanh(t) = 2 (t + t^3/3 + t^5/5 + ...),  t = (x-1)/(x+1),      */
/* |t| <= 0.1716, truncated after t^13 (remainder < 2^-27 relative).          */
/*   log u = e*ln2 + log x, with ln2 split in a 24-bit head and a tail.       */
/* Every operation is an IEEE single-precision operation in the order below.  */
/* ------------------------------------------------------------------------- */
static float f32_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_from_f32(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

float rxo_logf(float u)
{
    uint32_t b = bits_from_f32(u);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    float x = f32_from_bits((b & 0x007FFFFFu) | 0x3F800000u); /* [1, 2) */
    if (bits_from_f32(x) > 0x3FB504F3u) {                      /* x > sqrt(2) */
        x = x * 0.5f;
        e = e + 1;
    }
    float num = x - 1.0f;
    float den = x + 1.0f;
    float t = num / den;
    float t2 = t * t;
    /* coefficients 2/(2k+1), k = 1..6, each rounded to single precision */
    const float c3 = (float)(2.0 / 3.0), c5 = (float)(2.0 / 5.0), c7 = (float)(2.0 / 7.0);
    const float c9 = (float)(2.0 / 9.0), c11 = (float)(2.0 / 11.0), c13 = (float)(2.0 / 13.0);
    float p = c13;
    p = fmaf(p, t2, c11);
    p = fmaf(p, t2, c9);
    p = fmaf(p, t2, c7);
    p = fmaf(p, t2, c5);
    p = fmaf(p, t2, c3);
    float t3 = t * t2;
    float lx = fmaf(t3, p, t + t);
    /* ln 2 = LN2_HI + LN2_LO, LN2_HI = ln 2 rounded to single precision */
    const double ln2 = 0.693147180559945309417232121458;
    const float LN2_HI = (float)ln2;
    const float LN2_LO = (float)(ln2 - (double)LN2_HI);
    float fe = (float)e;
    return fmaf(fe, LN2_HI, fmaf(fe, LN2_LO, lx));
}

/* ------------------------------------------------------------------------- */
/* sin and cos of 2*pi*u for u = n * 2^-24, n in [1, 2^24], in FP32.          */
/* Exact range reduction in integers: 2*pi*u = (pi/2) (q + f) with            */
/* q = round(n / 2^22) and f = (n - q 2^22) 2^-22 in [-1/2, 1/2).             */
/* Then sin((pi/2) f), cos((pi/2) f) by their Taylor series in f              */
/* (coefficients (pi/2)^k / k!, truncated at f^9 and f^10), and the quadrant  */
/* q mod 4 rotates the pair.                                                  */
/* ------------------------------------------------------------------------- */
static double fact(int k) { double r = 1.0; for (int i = 2; i <= k; ++i) r *= i; return r; }

void rxo_sincos2pi(uint32_t n, float *s_out, float *c_out)
{
    const double hp = 1.57079632679489661923132169164; /* pi/2 */
    float S[5], C[6];
    for (int k = 0; k < 5; ++k) S[k] = (float)((k & 1 ? -1.0 : 1.0) * pow(hp, 2 * k + 1) / fact(2 * k + 1));
    for (int k = 0; k < 6; ++k) C[k] = (float)((k & 1 ? -1.0 : 1.0) * pow(hp, 2 * k) / fact(2 * k));
    int32_t q = (int32_t)((n + (1u << 21)) >> 22);   /* 0..4 */
    int32_t r = (int32_t)n - q * (int32_t)(1u << 22); /* [-2^21, 2^21) */
    float f = (float)r * 0x1p-22f;                     /* exact */
    float f2 = f * f;
    float sp = S[4];
    sp = fmaf(sp, f2, S[3]);
    sp = fmaf(sp, f2, S[2]);
    sp = fmaf(sp, f2, S[1]);
    float sn = fmaf(f * f2, sp, S[0] * f);
    float cp = C[5];
    cp = fmaf(cp, f2, C[4]);
    cp = fmaf(cp, f2, C[3]);
    cp = fmaf(cp, f2, C[2]);
    cp = fmaf(cp, f2, C[1]);
    float cs = fmaf(cp, f2, C[0]);
    switch (q & 3) {
    case 0: *s_out = sn; *c_out = cs; break;
    case 1: *s_out = cs; *c_out = -sn; break;
    case 2: *s_out = -sn; *c_out = -cs; break;
    default: *s_out = -cs; *c_out = sn; break;
    }
}

/* ------------------------------------------------------------------------- */
/* Standard normals for the Gaussian sketch (Section 2.3, "Gaussian           */
/* Ensemble").  Column i of Omega (i = row index of A) and rows 4k..4k+3 come */
/* from one Philox call with counter (i_lo, i_hi, k, stream) and key          */
/* (seed_lo, seed_hi).  Outputs x0..x3 become uniforms u = ((x>>8)+1) 2^-24   */
/* in (0,1], and Box-Muller turns (u0,u1) and (u2,u3) into                    */
/*   sqrt(-2 log u0) cos(2 pi u1), sqrt(-2 log u0) sin(2 pi u1), ...          */
/* ------------------------------------------------------------------------- */
void rxo_normal4(uint64_t seed, uint64_t i, uint32_t k, uint32_t stream, float z[4])
{
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), k, stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    rxo_philox4x32_10(ctr, key, x);
    for (int h = 0; h < 2; ++h) {
        uint32_t na = (x[2 * h] >> 8) + 1u, nb = (x[2 * h + 1] >> 8) + 1u;
        float ua = (float)na * 0x1p-24f;
        float lg = rxo_logf(ua);
        float rad = sqrtf(-2.0f * lg);
        float sn, cs;
        rxo_sincos2pi(nb, &sn, &cs);
        z[2 * h] = rad * cs;
        z[2 * h + 1] = rad * sn;
    }
}

/* z values of Omega for rows [i0, i0+rows) of A: z_out[(i-i0)*s + r], r < s. */
void rxo_omega_z(uint64_t seed, int64_t s, int64_t i0, int64_t rows, float *z_out)
{
    for (int64_t i = 0; i < rows; ++i) {
        for (int64_t k = 0; 4 * k < s; ++k) {
            float z[4];
            rxo_normal4(seed, (uint64_t)(i0 + i), (uint32_t)k, 0u, z);
            for (int t = 0; t < 4 && 4 * k + t < s; ++t) z_out[i * s + 4 * k + t] = z[t];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Sketch Y = Omega A (Section 2.3): Omega_{r,i} = c z_{r,i}, c = 1/sqrt(s),  */
/* entries N(0, 1/s).  Y_{r,j} = sum_i Omega_{r,i} A_{i,j}.  Rows of A are    */
/* summed in blocks of 256 and the block sums are combined pairwise (a binary */
/* counter of partial sums) so that the oracle's own rounding stays at        */
/* O(u log m).                                                                */
/* ------------------------------------------------------------------------- */
#define RXO_BLOCK 256

typedef struct {
    double *lev[64];
    int used[64];
    int64_t len;
} pairwise_t;

static void pw_init(pairwise_t *p, int64_t len)
{
    memset(p, 0, sizeof(*p));
    p->len = len;
}
static void pw_push(pairwise_t *p, const double *blk)
{
    /* carry like a binary counter: level L holds a sum of 2^L blocks */
    double *cur = (double *)malloc((size_t)p->len * sizeof(double));
    memcpy(cur, blk, (size_t)p->len * sizeof(double));
    int L = 0;
    while (p->used[L]) {
        for (int64_t t = 0; t < p->len; ++t) cur[t] = p->lev[L][t] + cur[t];
        free(p->lev[L]);
        p->lev[L] = NULL;
        p->used[L] = 0;
        ++L;
    }
    p->lev[L] = cur;
    p->used[L] = 1;
}
static void pw_finish(pairwise_t *p, double *out)
{
    int first = 1;
    for (int L = 0; L < 64; ++L) {
        if (!p->used[L]) continue;
        for (int64_t t = 0; t < p->len; ++t) out[t] = first ? p->lev[L][t] : p->lev[L][t] + out[t];
        first = 0;
        free(p->lev[L]);
        p->lev[L] = NULL;
        p->used[L] = 0;
    }
    if (first) memset(out, 0, (size_t)p->len * sizeof(double));
}

/* The split-precision sketch uses the same draws quantised to the 2^-12 grid,
 * z' = rint(4096 z) / 4096 (round half to even), so that each entry is two
 * 8-bit integers; quantise != 0 selects that matrix. */
static void sketch_impl(const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
                        int64_t row0, double *Y, int64_t ldy, int quantise);

void rxo_sketch(const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
                double *Y, int64_t ldy)
{
    sketch_impl(A, m, n, lda, s, seed, 0, Y, ldy, 0);
}

/* The sketch of a row shard: A holds rows row0 .. row0 + m - 1 of a larger
 * matrix and Omega's columns are those of the global rows (the row-block
 * partition of Section 2.4); the shards' sketches add up to the whole one. */
void rxo_sketch_shard(const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed, int64_t row0,
                      double *Y, int64_t ldy)
{
    sketch_impl(A, m, n, lda, s, seed, row0, Y, ldy, 0);
}

void rxo_sketch_quantised(const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
                          double *Y, int64_t ldy)
{
    sketch_impl(A, m, n, lda, s, seed, 0, Y, ldy, 1);
}

/* The partial sum of one 256-row block of Omega A (block rows b0 .. b0 + rows). */
static void sketch_block(const double *A, int64_t lda, int64_t n, int64_t s, uint64_t seed, int quantise, double c,
                         int64_t row0, int64_t b0, int64_t rows, float *z, double *blk)
{
    rxo_omega_z(seed, s, row0 + b0, rows, z);
    memset(blk, 0, (size_t)(s * n) * sizeof(double));
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double a = A[(b0 + i) + j * lda];
            for (int64_t r = 0; r < s; ++r) {
                double zr = (double)z[i * s + r];
                if (quantise) zr = nearbyint(zr * 4096.0) / 4096.0;
                double om = c * zr;
                blk[r + j * s] += om * a;
            }
        }
}

/* Blocks whose partial sums are formed side by side (then combined in order). */
#define RXO_BATCH 64

static void sketch_impl(const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
                        int64_t row0, double *Y, int64_t ldy, int quantise)
{
    const double c = 1.0 / sqrt((double)s);
    double *blk = (double *)malloc((size_t)(RXO_BATCH * s * n) * sizeof(double));
    pairwise_t pw;
    pw_init(&pw, s * n);
    const int64_t nblocks = (m + RXO_BLOCK - 1) / RXO_BLOCK;
    for (int64_t g0 = 0; g0 < nblocks; g0 += RXO_BATCH) {
        const int64_t nb = (nblocks - g0 < RXO_BATCH) ? nblocks - g0 : RXO_BATCH;
#pragma omp parallel
        {
            float *z = (float *)malloc((size_t)(s * RXO_BLOCK) * sizeof(float));
#pragma omp for schedule(dynamic, 1)
            for (int64_t q = 0; q < nb; ++q) {
                const int64_t b0 = (g0 + q) * RXO_BLOCK;
                const int64_t rows = (m - b0 < RXO_BLOCK) ? m - b0 : RXO_BLOCK;
                sketch_block(A, lda, n, s, seed, quantise, c, row0, b0, rows, z, blk + q * s * n);
            }
            free(z);
        }
        for (int64_t q = 0; q < nb; ++q) pw_push(&pw, blk + q * s * n);
    }
    pw_finish(&pw, blk);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t r = 0; r < s; ++r) Y[r + j * ldy] = blk[r + j * s];
    free(blk);
}

/* ------------------------------------------------------------------------- */
/* Row extraction (Section 2.3; Theorem 3.2's equal-probability case): the   */
/* submatrix A_1 = PA takes l rows of A chosen independently, each row i     */
/* with probability 1/m (with replacement), in draw order.  Draw k uses one  */
/* Philox4x32-10 call, counter (k_lo, k_hi, 0, 3), key (seed_lo, seed_hi):   */
/* u = out0 + 2^32 out1 is uniform on [0, 2^64), and the row is              */
/* floor(u m / 2^64) (exact in 128-bit integers).                            */
/* ------------------------------------------------------------------------- */
void rxo_row_indices(uint64_t seed, int64_t l, int64_t m, int64_t *idx)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t k = 0; k < l; ++k) {
        const uint32_t ctr[4] = {(uint32_t)k, (uint32_t)((uint64_t)k >> 32), 0u, 3u};
        uint32_t out[4];
        rxo_philox4x32_10(ctr, key, out);
        const uint64_t u = (uint64_t)out[0] | ((uint64_t)out[1] << 32);
        idx[k] = (int64_t)(((unsigned __int128)u * (unsigned __int128)(uint64_t)m) >> 64);
    }
}

/* Y (l x n, leading dimension ldy): row k of Y is row idx[k] of A. */
void rxo_sketch_rows(const double *A, int64_t m, int64_t n, int64_t lda, int64_t l, uint64_t seed, double *Y,
                     int64_t ldy)
{
    int64_t *idx = (int64_t *)malloc((size_t)l * sizeof(int64_t));
    rxo_row_indices(seed, l, m, idx);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t k = 0; k < l; ++k) Y[k + j * ldy] = A[idx[k] + j * lda];
    free(idx);
}

/* ------------------------------------------------------------------------- */
/* Householder Q-less QR of an l x n matrix (l >= n): the R factor of the    */
/* sketch, Algorithm 5 step 2.  Column k: x = W(k:l, k), alpha = ||x||,      */
/* v = x + sign(x_0) alpha e_1 (sign(0) = +1), beta = 2 / v^T v,            */
/* R_kk = -sign(x_0) alpha, and W(k:l, j) -= beta (v^T W(k:l, j)) v, j > k.  */
/* W is overwritten.  R (n x n) receives the upper triangle, zeros below.    */
/* ------------------------------------------------------------------------- */
void rxo_geqr_r(double *W, int64_t l, int64_t n, int64_t ldw, double *R, int64_t ldr)
{
    double *v = (double *)malloc((size_t)l * sizeof(double));
    for (int64_t k = 0; k < n; ++k) {
        double ss = 0.0;
        for (int64_t i = k; i < l; ++i) ss += W[i + k * ldw] * W[i + k * ldw];
        double alpha = sqrt(ss);
        double x0 = W[k + k * ldw];
        double sg = (x0 < 0.0) ? -1.0 : 1.0;
        for (int64_t i = k; i < l; ++i) v[i] = W[i + k * ldw];
        v[k] = x0 + sg * alpha;
        double vtv = 0.0;
        for (int64_t i = k; i < l; ++i) vtv += v[i] * v[i];
        W[k + k * ldw] = -sg * alpha;
        for (int64_t i = k + 1; i < l; ++i) W[i + k * ldw] = 0.0;
        if (vtv > 0.0) {
            double beta = 2.0 / vtv;
            for (int64_t j = k + 1; j < n; ++j) {
                double w = 0.0;
                for (int64_t i = k; i < l; ++i) w += v[i] * W[i + j * ldw];
                for (int64_t i = k; i < l; ++i) W[i + j * ldw] -= beta * w * v[i];
            }
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) R[i + j * ldr] = (i <= j) ? W[i + j * ldw] : 0.0;
    free(v);
}

/* ------------------------------------------------------------------------- */
/* LU with partial (row) pivoting of an l x n matrix (l >= n): the U factor, */
/* Algorithm 4 step 2.  Pivot = largest |entry| of the column at or below    */
/* the diagonal, the lowest row index on ties.  W is overwritten with L      */
/* (unit, below the diagonal) and U; piv[k] is the row swapped with k.       */
/* ------------------------------------------------------------------------- */
void rxo_getrf_u(double *W, int64_t l, int64_t n, int64_t ldw, double *U, int64_t ldu, int64_t *piv)
{
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        double best = fabs(W[k + k * ldw]);
        for (int64_t i = k + 1; i < l; ++i) {
            double a = fabs(W[i + k * ldw]);
            if (a > best) {
                best = a;
                p = i;
            }
        }
        if (piv) piv[k] = p;
        if (p != k)
            for (int64_t j = 0; j < n; ++j) {
                double t = W[k + j * ldw];
                W[k + j * ldw] = W[p + j * ldw];
                W[p + j * ldw] = t;
            }
        double d = W[k + k * ldw];
        if (d != 0.0) {
            for (int64_t i = k + 1; i < l; ++i) {
                double lik = W[i + k * ldw] / d;
                W[i + k * ldw] = lik;
                for (int64_t j = k + 1; j < n; ++j) W[i + j * ldw] -= lik * W[k + j * ldw];
            }
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) U[i + j * ldu] = (i <= j) ? W[i + j * ldw] : 0.0;
}

/* Scale row k of the upper-triangular R by sign(R_kk) so that diag(R) >= 0.  */
void rxo_sign_normalise(double *R, int64_t n, int64_t ldr)
{
    for (int64_t k = 0; k < n; ++k)
        if (R[k + k * ldr] < 0.0)
            for (int64_t j = k; j < n; ++j) R[k + j * ldr] = -R[k + j * ldr];
}

/* Singular sketch factor: a non-finite diagonal, or |R_kk| <= n u max|R_jj|  */
/* with u = 2^-53 (a rank-deficient sketch, Section 2.2).                     */
int rxo_check_factor(const double *R, int64_t n, int64_t ldr)
{
    double mx = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        double d = fabs(R[k + k * ldr]);
        if (!isfinite(d)) return RXO_SKETCH_SINGULAR;
        if (d > mx) mx = d;
    }
    double tol = (double)n * ldexp(1.0, -53) * mx;
    for (int64_t k = 0; k < n; ++k)
        if (!(fabs(R[k + k * ldr]) > tol)) return RXO_SKETCH_SINGULAR;
    return RXO_OK;
}

/* ------------------------------------------------------------------------- */
/* X = A R^{-1} for upper-triangular R, row by row by forward substitution   */
/* (x R = a): x_j = (a_j - sum_{k<j} x_k R_kj) / R_jj.  This is the           */
/* "solve a triangular system" step of Algorithm 1 and steps 3 of             */
/* Algorithms 4 and 5.  X may alias A (same leading dimension).               */
/* ------------------------------------------------------------------------- */
void rxo_trsm_right_upper(const double *A, int64_t m, int64_t n, int64_t lda, const double *R, int64_t ldr,
                          double *X, int64_t ldx)
{
#pragma omp parallel
    {
        double *x = (double *)malloc((size_t)n * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m; ++i) {
            for (int64_t j = 0; j < n; ++j) {
                double acc = A[i + j * lda];
                for (int64_t k = 0; k < j; ++k) acc -= x[k] * R[k + j * ldr];
                x[j] = acc / R[j + j * ldr];
            }
            for (int64_t j = 0; j < n; ++j) X[i + j * ldx] = x[j];
        }
        free(x);
    }
}

/* G = X^T X (n x n, full symmetric), Algorithm 1 step 1; 256-row blocks     */
/* combined pairwise as in the sketch.                                        */
void rxo_gram(const double *X, int64_t m, int64_t n, int64_t ldx, double *G, int64_t ldg)
{
    double *blk = (double *)malloc((size_t)(RXO_BATCH * n * n) * sizeof(double));
    pairwise_t pw;
    pw_init(&pw, n * n);
    const int64_t nblocks = (m + RXO_BLOCK - 1) / RXO_BLOCK;
    for (int64_t g0 = 0; g0 < nblocks; g0 += RXO_BATCH) {
        const int64_t nb = (nblocks - g0 < RXO_BATCH) ? nblocks - g0 : RXO_BATCH;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t q = 0; q < nb; ++q) {
            const int64_t b0 = (g0 + q) * RXO_BLOCK;
            const int64_t rows = (m - b0 < RXO_BLOCK) ? m - b0 : RXO_BLOCK;
            double *bq = blk + q * n * n;
            memset(bq, 0, (size_t)(n * n) * sizeof(double));
            for (int64_t j = 0; j < n; ++j)
                for (int64_t l = 0; l <= j; ++l) {
                    double acc = 0.0;
                    for (int64_t i = b0; i < b0 + rows; ++i) acc += X[i + l * ldx] * X[i + j * ldx];
                    bq[l + j * n] = acc;
                }
        }
        for (int64_t q = 0; q < nb; ++q) pw_push(&pw, blk + q * n * n);
    }
    pw_finish(&pw, blk);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t l = 0; l <= j; ++l) {
            G[l + j * ldg] = blk[l + j * n];
            G[j + l * ldg] = blk[l + j * n];
        }
    free(blk);
}

/* ------------------------------------------------------------------------- */
/* Upper Cholesky factor, Algorithm 1 step 2: R^T R = G, reading only the    */
/* upper triangle of G.  R_jj = sqrt(G_jj - sum_{k<j} R_kj^2),               */
/* R_jl = (G_jl - sum_{k<j} R_kj R_kl) / R_jj.  Returns 0, or j+1 when the   */
/* argument of the square root in column j is not positive or not finite     */
/* (breakdown, Section 2.1).                                                  */
/* ------------------------------------------------------------------------- */
int rxo_potrf_u(const double *G, int64_t n, int64_t ldg, double *R, int64_t ldr)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) R[i + j * ldr] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double d = G[j + j * ldg];
        for (int64_t k = 0; k < j; ++k) d -= R[k + j * ldr] * R[k + j * ldr];
        if (!(d > 0.0) || !isfinite(d)) return (int)(j + 1);
        double rjj = sqrt(d);
        R[j + j * ldr] = rjj;
        for (int64_t l = j + 1; l < n; ++l) {
            double a = G[j + l * ldg];
            for (int64_t k = 0; k < j; ++k) a -= R[k + j * ldr] * R[k + l * ldr];
            R[j + l * ldr] = a / rjj;
        }
    }
    return 0;
}

/* C = A B for upper-triangular A, B (n x n); C may not alias A or B. */
void rxo_trmm_upper(const double *A, int64_t lda, const double *B, int64_t ldb, int64_t n, double *C, int64_t ldc)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) {
            double acc = 0.0;
            if (i <= j)
                for (int64_t k = i; k <= j; ++k) acc += A[i + k * lda] * B[k + j * ldb];
            C[i + j * ldc] = acc;
        }
}

static int all_finite(const double *A, int64_t m, int64_t n, int64_t lda)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i)
            if (!isfinite(A[i + j * lda])) return 0;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* rLU- / rQR-CholeskyQR (Algorithms 4 and 5; Algorithm A.1 is what is       */
/* computed in floating point), with the CholeskyQR step repeated `passes`    */
/* times as in CholeskyQR2 (Algorithm 2):                                     */
/*   1  Y = Omega A (Gaussian sketch, s rows)                                 */
/*   2  R_s = R factor of Y by LU (variant LU) or Householder QR (variant QR),*/
/*      rows scaled so that diag(R_s) > 0                                     */
/*   3  X = A R_s^{-1}                                                        */
/*   4  for p = 1..passes: G = X^T X, R_p = chol(G), X = X R_p^{-1}           */
/*   5  Q = X, R = R_passes ... R_1 R_s                                       */
/* Variant NONE takes R_s = I (plain CholeskyQR / CholeskyQR2).  LU or QR    */
/* with RXO_SKETCH_ROWS takes the sketch by row extraction.                  */
/* Optional outputs (NULL to skip): Y (s x n, ld s), Rs (n x n), G1, R1      */
/* (n x n, the first pass), G2, R2 (the second pass), info = breakdown pass  */
/* and column.                                                                */
/* ------------------------------------------------------------------------- */
int rxo_rxr_cholqr(const double *A, int64_t m, int64_t n, int64_t lda, int variant, int64_t s, uint64_t seed,
                   int passes, double *Q, int64_t ldq, double *R, int64_t ldr, double *Y_out, double *Rs_out,
                   double *G1_out, double *R1_out, double *G2_out, double *R2_out, int *info)
{
    if (info) {
        info[0] = 0;
        info[1] = 0;
    }
    if (!all_finite(A, m, n, lda)) return RXO_NONFINITE;
    size_t nn = (size_t)(n * n);
    double *Rs = (double *)calloc(nn, sizeof(double));
    double *Racc = (double *)calloc(nn, sizeof(double));
    double *tmp = (double *)calloc(nn, sizeof(double));
    double *G = (double *)calloc(nn, sizeof(double));
    double *Rp = (double *)calloc(nn, sizeof(double));
    int status = RXO_OK;

    const int rows = (variant & RXO_SKETCH_ROWS) != 0;
    variant &= ~RXO_SKETCH_ROWS;
    if (variant == RXO_VARIANT_NONE) {
        for (int64_t k = 0; k < n; ++k) Rs[k + k * n] = 1.0;
    } else {
        double *Y = (double *)malloc((size_t)(s * n) * sizeof(double));
        if (rows)
            rxo_sketch_rows(A, m, n, lda, s, seed, Y, s);
        else
            rxo_sketch(A, m, n, lda, s, seed, Y, s);
        if (Y_out) memcpy(Y_out, Y, (size_t)(s * n) * sizeof(double));
        if (variant == RXO_VARIANT_QR)
            rxo_geqr_r(Y, s, n, s, Rs, n);
        else
            rxo_getrf_u(Y, s, n, s, Rs, n, NULL);
        free(Y);
        rxo_sign_normalise(Rs, n, n);
        status = rxo_check_factor(Rs, n, n);
    }
    if (Rs_out) memcpy(Rs_out, Rs, nn * sizeof(double));
    if (status == RXO_OK) {
        rxo_trsm_right_upper(A, m, n, lda, Rs, n, Q, ldq);
        memcpy(Racc, Rs, nn * sizeof(double));
        for (int p = 1; p <= passes; ++p) {
            rxo_gram(Q, m, n, ldq, G, n);
            int bad = rxo_potrf_u(G, n, n, Rp, n);
            if (p == 1 && G1_out) memcpy(G1_out, G, nn * sizeof(double));
            if (p == 2 && G2_out) memcpy(G2_out, G, nn * sizeof(double));
            if (bad) {
                status = RXO_CHOL_BREAKDOWN;
                if (info) {
                    info[0] = p;
                    info[1] = bad - 1;
                }
                break;
            }
            if (p == 1 && R1_out) memcpy(R1_out, Rp, nn * sizeof(double));
            if (p == 2 && R2_out) memcpy(R2_out, Rp, nn * sizeof(double));
            rxo_trsm_right_upper(Q, m, n, ldq, Rp, n, Q, ldq);
            rxo_trmm_upper(Rp, n, Racc, n, n, tmp, n);
            memcpy(Racc, tmp, nn * sizeof(double));
        }
        if (status == RXO_OK && R)
            for (int64_t j = 0; j < n; ++j)
                for (int64_t i = 0; i < n; ++i) R[i + j * ldr] = Racc[i + j * n];
    }
    free(Rs);
    free(Racc);
    free(tmp);
    free(G);
    free(Rp);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Least squares preconditioned by the sketch's R factor (Section 5.2):      */
/*   1  B = A R_s^{-1}  (R_s from the sketch: rQR / rLU, Gaussian or rows)    */
/*   2  y = (B^T B)^{-1} B^T b  by the normal equations: G = B^T B,           */
/*      R_G = chol(G), c = B^T b, R_G^T z = c, R_G y = z                      */
/*   3  x = R_s^{-1} y                                                        */
/* b is m x k (ldb), x is n x k (ldx).  Returns the status of the sketch's   */
/* factor, of the Cholesky step, or NONFINITE for A or b.                    */
/* ------------------------------------------------------------------------- */
int rxo_lstsq(const double *A, int64_t m, int64_t n, int64_t lda, const double *b, int64_t k, int64_t ldb, int variant,
              int64_t s, uint64_t seed, double *x, int64_t ldx)
{
    if (!all_finite(A, m, n, lda) || !all_finite(b, m, k, ldb)) return RXO_NONFINITE;
    const int rows = (variant & RXO_SKETCH_ROWS) != 0;
    variant &= ~RXO_SKETCH_ROWS;
    size_t nn = (size_t)(n * n);
    double *Y = (double *)malloc((size_t)(s * n) * sizeof(double));
    double *Rs = (double *)calloc(nn, sizeof(double));
    double *G = (double *)calloc(nn, sizeof(double));
    double *RG = (double *)calloc(nn, sizeof(double));
    double *B = (double *)malloc((size_t)(m * n) * sizeof(double));
    double *c = (double *)malloc((size_t)n * sizeof(double));
    int status = RXO_OK;
    if (rows)
        rxo_sketch_rows(A, m, n, lda, s, seed, Y, s);
    else
        rxo_sketch(A, m, n, lda, s, seed, Y, s);
    if (variant == RXO_VARIANT_QR)
        rxo_geqr_r(Y, s, n, s, Rs, n);
    else
        rxo_getrf_u(Y, s, n, s, Rs, n, NULL);
    rxo_sign_normalise(Rs, n, n);
    status = rxo_check_factor(Rs, n, n);
    if (status == RXO_OK) {
        rxo_trsm_right_upper(A, m, n, lda, Rs, n, B, m);
        rxo_gram(B, m, n, m, G, n);
        if (rxo_potrf_u(G, n, n, RG, n)) status = RXO_CHOL_BREAKDOWN;
    }
    for (int64_t r = 0; status == RXO_OK && r < k; ++r) {
        const double *br = b + r * ldb;
        double *xr = x + r * ldx;
        for (int64_t j = 0; j < n; ++j) { /* c = B^T b */
            double acc = 0.0;
            for (int64_t i = 0; i < m; ++i) acc += B[i + j * m] * br[i];
            c[j] = acc;
        }
        for (int64_t j = 0; j < n; ++j) { /* R_G^T z = c (forward) */
            double acc = c[j];
            for (int64_t l = 0; l < j; ++l) acc -= RG[l + j * n] * c[l];
            c[j] = acc / RG[j + j * n];
        }
        for (int64_t j = n - 1; j >= 0; --j) { /* R_G y = z (backward) */
            double acc = c[j];
            for (int64_t l = j + 1; l < n; ++l) acc -= RG[j + l * n] * c[l];
            c[j] = acc / RG[j + j * n];
        }
        for (int64_t j = n - 1; j >= 0; --j) { /* R_s x = y (backward) */
            double acc = c[j];
            for (int64_t l = j + 1; l < n; ++l) acc -= Rs[j + l * n] * xr[l];
            xr[j] = acc / Rs[j + j * n];
        }
    }
    free(Y);
    free(Rs);
    free(G);
    free(RG);
    free(B);
    free(c);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Shifted CholeskyQR3 (the comparator of Section 2.1's algorithm            */
/* sCholeskyQR3): G = A^T A, R_1 = chol(G + shift I), Q_1 = A R_1^{-1}, then */
/* passes - 1 plain CholeskyQR steps (two for sCholeskyQR3), R = R_p ... R_1. */
/* The shift is an input (absolute).  info = breakdown pass and column.      */
/* ------------------------------------------------------------------------- */
int rxo_scholqr(const double *A, int64_t m, int64_t n, int64_t lda, double shift, int passes, double *Q,
                int64_t ldq, double *R, int64_t ldr, int *info)
{
    if (info) {
        info[0] = 0;
        info[1] = 0;
    }
    if (!all_finite(A, m, n, lda)) return RXO_NONFINITE;
    size_t nn = (size_t)(n * n);
    double *Racc = (double *)calloc(nn, sizeof(double));
    double *tmp = (double *)calloc(nn, sizeof(double));
    double *G = (double *)calloc(nn, sizeof(double));
    double *Rp = (double *)calloc(nn, sizeof(double));
    int status = RXO_OK;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) Q[i + j * ldq] = A[i + j * lda];
    for (int64_t k = 0; k < n; ++k) Racc[k + k * n] = 1.0;
    for (int p = 1; p <= passes; ++p) {
        rxo_gram(Q, m, n, ldq, G, n);
        if (p == 1)
            for (int64_t k = 0; k < n; ++k) G[k + k * n] += shift;
        int bad = rxo_potrf_u(G, n, n, Rp, n);
        if (bad) {
            status = RXO_CHOL_BREAKDOWN;
            if (info) {
                info[0] = p;
                info[1] = bad - 1;
            }
            break;
        }
        rxo_trsm_right_upper(Q, m, n, ldq, Rp, n, Q, ldq);
        rxo_trmm_upper(Rp, n, Racc, n, n, tmp, n);
        memcpy(Racc, tmp, nn * sizeof(double));
    }
    if (status == RXO_OK && R)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) R[i + j * ldr] = Racc[i + j * n];
    free(Racc);
    free(tmp);
    free(G);
    free(Rp);
    return status;
}

/* ------------------------------------------------------------------------- */
/* The plain definition of the result: the thin QR factorisation A = QR with */
/* diag(R) > 0, which is unique for full-rank A (footnote to Algorithm 1).   */
/* Householder QR of A (copied), then Q = H_1 ... H_n [I; 0] accumulated     */
/* backwards, then rows of R and columns of Q with R_kk < 0 flip sign.       */
/* ------------------------------------------------------------------------- */
void rxo_householder_qr(const double *A, int64_t m, int64_t n, int64_t lda, double *Q, int64_t ldq, double *R,
                        int64_t ldr)
{
    double *W = (double *)malloc((size_t)(m * n) * sizeof(double));
    double *V = (double *)malloc((size_t)(m * n) * sizeof(double)); /* reflectors */
    double *beta = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) W[i + j * m] = A[i + j * lda];
    for (int64_t k = 0; k < n; ++k) {
        double ss = 0.0;
        for (int64_t i = k; i < m; ++i) ss += W[i + k * m] * W[i + k * m];
        double alpha = sqrt(ss);
        double x0 = W[k + k * m];
        double sg = (x0 < 0.0) ? -1.0 : 1.0;
        for (int64_t i = 0; i < m; ++i) V[i + k * m] = (i < k) ? 0.0 : W[i + k * m];
        V[k + k * m] = x0 + sg * alpha;
        double vtv = 0.0;
        for (int64_t i = k; i < m; ++i) vtv += V[i + k * m] * V[i + k * m];
        beta[k] = (vtv > 0.0) ? 2.0 / vtv : 0.0;
        W[k + k * m] = -sg * alpha;
        for (int64_t i = k + 1; i < m; ++i) W[i + k * m] = 0.0;
        for (int64_t j = k + 1; j < n; ++j) {
            double w = 0.0;
            for (int64_t i = k; i < m; ++i) w += V[i + k * m] * W[i + j * m];
            for (int64_t i = k; i < m; ++i) W[i + j * m] -= beta[k] * w * V[i + k * m];
        }
    }
    /* Q = H_0 H_1 ... H_{n-1} [I; 0] */
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) Q[i + j * ldq] = (i == j) ? 1.0 : 0.0;
    for (int64_t k = n - 1; k >= 0; --k)
        for (int64_t j = 0; j < n; ++j) {
            double w = 0.0;
            for (int64_t i = k; i < m; ++i) w += V[i + k * m] * Q[i + j * ldq];
            for (int64_t i = k; i < m; ++i) Q[i + j * ldq] -= beta[k] * w * V[i + k * m];
        }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) R[i + j * ldr] = (i <= j) ? W[i + j * m] : 0.0;
    for (int64_t k = 0; k < n; ++k)
        if (R[k + k * ldr] < 0.0) {
            for (int64_t j = k; j < n; ++j) R[k + j * ldr] = -R[k + j * ldr];
            for (int64_t i = 0; i < m; ++i) Q[i + k * ldq] = -Q[i + k * ldq];
        }
    free(W);
    free(V);
    free(beta);
}

/* ------------------------------------------------------------------------- */
/* Accuracy measures of Section 4.2, evaluated with compensated dot products  */
/* (Ogita, Rump & Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. */
/* 2005, algorithm Dot2: TwoProduct by fma, TwoSum by Knuth), so that the     */
/* evaluation error is far below the quantities measured.                     */
/* ------------------------------------------------------------------------- */
typedef struct {
    double p, s;
} dot2_t;
static void dot2_add(dot2_t *d, double x, double y)
{
    double h = x * y;
    double r = fma(x, y, -h);
    double p = d->p + h;
    double z = p - d->p;
    double q = (d->p - (p - z)) + (h - z);
    d->p = p;
    d->s += q + r;
}

/* ||Q^T Q - I||_F */
double rxo_orth_error(const double *Q, int64_t m, int64_t n, int64_t ldq)
{
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t l = 0; l < n; ++l) {
            dot2_t d = {0.0, 0.0};
            if (j == l) dot2_add(&d, -1.0, 1.0);
            for (int64_t i = 0; i < m; ++i) dot2_add(&d, Q[i + j * ldq], Q[i + l * ldq]);
            double e = d.p + d.s;
            acc += e * e;
        }
    return sqrt(acc);
}

/* ||A - QR||_F / ||A||_F, R upper triangular */
double rxo_resid_error(const double *A, int64_t m, int64_t n, int64_t lda, const double *Q, int64_t ldq,
                       const double *R, int64_t ldr)
{
    double num = 0.0, den = 0.0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) {
            dot2_t d = {0.0, 0.0};
            dot2_add(&d, A[i + j * lda], 1.0);
            for (int64_t k = 0; k <= j; ++k) dot2_add(&d, -Q[i + k * ldq], R[k + j * ldr]);
            double e = d.p + d.s;
            num += e * e;
            den += A[i + j * lda] * A[i + j * lda];
        }
    return sqrt(num) / sqrt(den);
}

/* Compensated dot product, exposed so that tests can pin Dot2 itself. */
double rxo_dot2(const double *x, const double *y, int64_t len)
{
    dot2_t d = {0.0, 0.0};
    for (int64_t i = 0; i < len; ++i) dot2_add(&d, x[i], y[i]);
    return d.p + d.s;
}
