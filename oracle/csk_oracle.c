/*
 * csk_oracle.c -- plain CPU oracle of the Count Sketch Kaczmarz method
 * (arXiv 2004.02480).  TEST INFRASTRUCTURE ONLY: used by the tests, the smoke
 * check and the benchmark's CPU-baseline leg; never by the product path.
 *
 * Everything here is written for a reader checking it against the paper:
 * no blocking, no fusion, no reordering beyond what each docstring states.
 * Function-by-function citations:
 *   or_count_sketch_map   Definition 1 (count sketch transform S = Phi D)
 *   or_stable_count_sort  not in the paper; the order Definition 1 leaves
 *                         free is fixed as ascending row index
 *   or_sketch_*           Algorithm 1, "Initialize" (At = S A, bt = S b)
 *   or_mwrk               Algorithm 1, loop steps (selection rule and
 *                         projection); stopping rule of Section 3
 *   or_csk                Algorithm 1 as a whole; d == 0 is the MWRK method
 *                         of Remark 1
 *   or_final_check        RES of Section 3 and the sketched residual
 *   or_gram_*             G = At At^T, the matrix whose columns give the
 *                         residual change r_{k+1} = r_k - alpha G e_{i_k},
 *                         which follows from the update of Algorithm 1
 */
#include "csk_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- hashing */

uint64_t or_splitmix64_at(uint64_t seed, uint64_t c)
{
    /* SplitMix64: the state advances by the golden-ratio increment and each
     * output is the state passed through the 64-bit finaliser. */
    uint64_t z = seed + c * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void or_count_sketch_map(uint64_t seed, int64_t m, int64_t d,
                         int32_t *h, int8_t *sign)
{
    for (int64_t i = 0; i < m; ++i) {
        uint64_t u = or_splitmix64_at(seed, (uint64_t)i + 1u);
        /* h(i) = j with probability 1/d: multiply-shift reduction of a
         * uniform 32-bit value onto [0, d). */
        uint64_t hi32 = u >> 32;
        if (h) h[i] = (int32_t)((hi32 * (uint64_t)d) >> 32);
        /* D_ii = +1 or -1 with equal probability. */
        if (sign) sign[i] = (u & 1u) ? (int8_t)-1 : (int8_t)1;
    }
}

/* ------------------------------------------------------ counting sort */

void or_stable_count_sort(const int32_t *h, int64_t m, int64_t d,
                          int32_t *cnt, int32_t *off, int32_t *perm)
{
    int32_t *c = (int32_t *)calloc((size_t)d, sizeof(int32_t));
    int32_t *o = (int32_t *)calloc((size_t)d + 1, sizeof(int32_t));
    int32_t *next = (int32_t *)calloc((size_t)d, sizeof(int32_t));
    for (int64_t i = 0; i < m; ++i) c[h[i]] += 1;
    o[0] = 0;
    for (int64_t j = 0; j < d; ++j) o[j + 1] = o[j] + c[j];
    for (int64_t j = 0; j < d; ++j) next[j] = o[j];
    if (perm) {
        for (int64_t i = 0; i < m; ++i) {      /* ascending i: stable */
            perm[next[h[i]]] = (int32_t)i;
            next[h[i]] += 1;
        }
    }
    if (cnt) memcpy(cnt, c, (size_t)d * sizeof(int32_t));
    if (off) memcpy(off, o, ((size_t)d + 1) * sizeof(int32_t));
    free(c); free(o); free(next);
}

/* ------------------------------------------------------------- sketch */

void or_sketch_f64(const double *A, int64_t m, int64_t n, int64_t lda,
                   const double *B, int64_t ldb, int64_t nrhs,
                   const int32_t *h, const int8_t *sign, int64_t d,
                   double *At, double *bt)
{
    memset(At, 0, (size_t)(d * n) * sizeof(double));
    if (B && bt) memset(bt, 0, (size_t)(d * nrhs) * sizeof(double));
    /* Column i of S has the single entry D_ii at row h(i), so row j of S A
     * is the signed sum of the rows of A mapped to bucket j. */
    for (int64_t i = 0; i < m; ++i) {
        double s = (double)sign[i];
        double *dst = At + (int64_t)h[i] * n;
        const double *src = A + i * lda;
        for (int64_t c = 0; c < n; ++c) dst[c] += s * src[c];
        if (B && bt) {
            double *bd = bt + (int64_t)h[i] * nrhs;
            const double *bs = B + i * ldb;
            for (int64_t r = 0; r < nrhs; ++r) bd[r] += s * bs[r];
        }
    }
}

void or_sketch_f32_same_order(const float *A, int64_t m, int64_t n,
                              int64_t lda, const float *B, int64_t ldb,
                              int64_t nrhs, const int32_t *h,
                              const int8_t *sign, int64_t d,
                              float *At, float *bt)
{
    memset(At, 0, (size_t)(d * n) * sizeof(float));
    if (B && bt) memset(bt, 0, (size_t)(d * nrhs) * sizeof(float));
    for (int64_t i = 0; i < m; ++i) {
        float *dst = At + (int64_t)h[i] * n;
        const float *src = A + i * lda;
        for (int64_t c = 0; c < n; ++c) {
            /* one binary32 addition (or subtraction) per term */
            volatile float t = (sign[i] > 0) ? dst[c] + src[c] : dst[c] - src[c];
            dst[c] = t;
        }
        if (B && bt) {
            float *bd = bt + (int64_t)h[i] * nrhs;
            const float *bs = B + i * ldb;
            for (int64_t r = 0; r < nrhs; ++r) {
                volatile float t = (sign[i] > 0) ? bd[r] + bs[r] : bd[r] - bs[r];
                bd[r] = t;
            }
        }
    }
}

void or_row_norms2_f64(const double *At, int64_t d, int64_t n, int64_t ld,
                       double *N)
{
    for (int64_t j = 0; j < d; ++j) {
        double s = 0.0;
        for (int64_t c = 0; c < n; ++c) s += At[j * ld + c] * At[j * ld + c];
        N[j] = s;
    }
}

void or_row_norms2_of_f32(const float *At, int64_t d, int64_t n, int64_t ld,
                          double *N)
{
    for (int64_t j = 0; j < d; ++j) {
        double s = 0.0;
        for (int64_t c = 0; c < n; ++c) {
            double v = (double)At[j * ld + c];
            s += v * v;
        }
        N[j] = s;
    }
}

/* ----------------------------------------------------------- iteration */

static double sq_dist(const double *x, const double *y, int64_t n)
{
    double s = 0.0;
    for (int64_t c = 0; c < n; ++c) {
        double t = x[c] - y[c];
        s += t * t;
    }
    return s;
}

static double sq_norm(const double *x, int64_t n)
{
    double s = 0.0;
    for (int64_t c = 0; c < n; ++c) s += x[c] * x[c];
    return s;
}

/* r = bt - At x, one sequential dot product per row. */
static void residual(const double *At, const double *bt, int64_t d,
                     int64_t n, int64_t ld, const double *x, double *r,
                     int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
#endif
    for (int64_t j = 0; j < d; ++j) {
        double s = 0.0;
        const double *row = At + j * ld;
        for (int64_t c = 0; c < n; ++c) s += row[c] * x[c];
        r[j] = bt[j] - s;
    }
#ifndef _OPENMP
    (void)nthreads;
#endif
}

int or_mwrk(const double *At, const double *bt, int64_t d, int64_t n,
            int64_t ld, const double *x0, const double *x_star, double tol,
            int64_t max_iter, int nthreads, double *x, int64_t *iters,
            int64_t log_len, int32_t *ik_log, double *gap_log,
            double *err2_log, double *rik_log, double *nik_log)
{
    double *N = (double *)malloc((size_t)d * sizeof(double));
    double *r = (double *)malloc((size_t)d * sizeof(double));
    int status = 0;
    int64_t k = 0;

    or_row_norms2_f64(At, d, n, ld, N);
    int any_row = 0;
    for (int64_t j = 0; j < d; ++j) if (N[j] > 0.0) any_row = 1;

    for (int64_t c = 0; c < n; ++c) x[c] = x0 ? x0[c] : 0.0;
    double xs2 = x_star ? sq_norm(x_star, n) : 0.0;
    double bt2 = sq_norm(bt, d);

    if (!any_row) { status = -4; goto done; }

    for (;;) {
        residual(At, bt, d, n, ld, x, r, nthreads);

        /* stopping rule, tested before the step (Section 3) */
        double err2 = x_star ? sq_dist(x, x_star, n) : 0.0;
        if (k < log_len && err2_log) err2_log[k] = err2;
        if (x_star) {
            if (err2 / xs2 <= tol) break;
        } else {
            if (sq_norm(r, d) / bt2 <= tol) break;
        }
        if (k >= max_iter) { status = 1; break; }

        /* selection: i_k = argmax |r_j| / ||At_j|| over non-zero rows */
        int64_t best = -1;
        double t1 = -1.0, t2 = -1.0;
        for (int64_t j = 0; j < d; ++j) {
            if (!(N[j] > 0.0)) continue;
            double w = fabs(r[j]) / sqrt(N[j]);
            if (isnan(w)) { status = -4; goto done; }
            if (w > t1) { t2 = t1; t1 = w; best = j; }
            else if (w > t2) { t2 = w; }
        }
        if (k < log_len) {
            if (ik_log) ik_log[k] = (int32_t)best;
            if (gap_log) gap_log[k] = (t2 >= 0.0 && t1 > 0.0) ? (t1 - t2) / t1 : 0.0;
            if (rik_log) rik_log[k] = r[best];
            if (nik_log) nik_log[k] = N[best];
        }
        if (t1 == 0.0) break;                 /* every residual is exactly 0 */

        /* projection onto the hyperplane of row i_k */
        double alpha = r[best] / N[best];
        const double *row = At + best * ld;
        for (int64_t c = 0; c < n; ++c) x[c] += alpha * row[c];
        k += 1;
    }
done:
    if (iters) *iters = k;
    free(N); free(r);
    return status;
}

int or_csk(const double *A, const double *b, int64_t m, int64_t n,
           int64_t lda, int64_t d, uint64_t seed, const double *x0,
           const double *x_star, double tol, int64_t max_iter, int nthreads,
           double *x, int64_t *iters)
{
    if (d == 0) {
        /* Remark 1: MWRK is Algorithm 1 with S = I. */
        return or_mwrk(A, b, m, n, lda, x0, x_star, tol, max_iter, nthreads,
                       x, iters, 0, NULL, NULL, NULL, NULL, NULL);
    }
    int32_t *h = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    int8_t *sg = (int8_t *)malloc((size_t)m);
    double *At = (double *)malloc((size_t)(d * n) * sizeof(double));
    double *bt = (double *)malloc((size_t)d * sizeof(double));
    or_count_sketch_map(seed, m, d, h, sg);
    or_sketch_f64(A, m, n, lda, b, 1, 1, h, sg, d, At, bt);
    int st = or_mwrk(At, bt, d, n, n, x0, x_star, tol, max_iter, nthreads, x,
                     iters, 0, NULL, NULL, NULL, NULL, NULL);
    free(h); free(sg); free(At); free(bt);
    return st;
}

void or_final_check(const double *At, const double *bt, int64_t d, int64_t n,
                    int64_t ld, const double *x, const double *x_star,
                    double *rse, double *resid)
{
    double *r = (double *)malloc((size_t)d * sizeof(double));
    residual(At, bt, d, n, ld, x, r, 1);
    if (resid) *resid = sqrt(sq_norm(r, d) / sq_norm(bt, d));
    if (rse) *rse = x_star ? sq_dist(x, x_star, n) / sq_norm(x_star, n) : NAN;
    free(r);
}

/* ---------------------------------------------------------------- Gram */

float or_bf16_round(float v)
{
    /* keep the top 16 bits of the binary32 pattern, rounding the dropped 16
     * bits to nearest with ties to even */
    uint32_t u;
    memcpy(&u, &v, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7FFFu + lsb) & 0xFFFF0000u;
    float out;
    memcpy(&out, &u, 4);
    return out;
}

void or_gram_f64(const double *At, int64_t d, int64_t n, int64_t ld,
                 double *G)
{
    for (int64_t i = 0; i < d; ++i)
        for (int64_t j = 0; j < d; ++j) {
            double s = 0.0;
            for (int64_t c = 0; c < n; ++c) s += At[i * ld + c] * At[j * ld + c];
            G[i * d + j] = s;
        }
}

void or_gram_split_bf16(const float *At, int64_t d, int64_t n, int64_t ld,
                        double *G)
{
    double *hi = (double *)malloc((size_t)(d * n) * sizeof(double));
    double *lo = (double *)malloc((size_t)(d * n) * sizeof(double));
    for (int64_t i = 0; i < d; ++i)
        for (int64_t c = 0; c < n; ++c) {
            float a = At[i * ld + c];
            float h = or_bf16_round(a);
            float l = or_bf16_round(a - h);   /* a - h is exact in binary32 */
            hi[i * n + c] = (double)h;
            lo[i * n + c] = (double)l;
        }
    for (int64_t i = 0; i < d; ++i)
        for (int64_t j = 0; j < d; ++j) {
            double s = 0.0;
            for (int64_t c = 0; c < n; ++c) {
                s += hi[i * n + c] * hi[j * n + c];
                s += hi[i * n + c] * lo[j * n + c];
                s += lo[i * n + c] * hi[j * n + c];
            }
            G[i * d + j] = s;
        }
    free(hi); free(lo);
}

void or_gram_split_bf16_rows(const float *At, int64_t d, int64_t n, int64_t ld,
                             const int64_t *rows, int64_t nrows, double *Grows)
{
    double *hi = (double *)malloc((size_t)(d * n) * sizeof(double));
    double *lo = (double *)malloc((size_t)(d * n) * sizeof(double));
    for (int64_t i = 0; i < d; ++i)
        for (int64_t c = 0; c < n; ++c) {
            float a = At[i * ld + c];
            float h = or_bf16_round(a);
            float l = or_bf16_round(a - h);
            hi[i * n + c] = (double)h;
            lo[i * n + c] = (double)l;
        }
    for (int64_t q = 0; q < nrows; ++q) {
        int64_t i = rows[q];
        for (int64_t j = 0; j < d; ++j) {
            double s = 0.0;
            for (int64_t c = 0; c < n; ++c) {
                s += hi[i * n + c] * hi[j * n + c];
                s += hi[i * n + c] * lo[j * n + c];
                s += lo[i * n + c] * hi[j * n + c];
            }
            Grows[q * d + j] = s;
        }
    }
    free(hi); free(lo);
}
