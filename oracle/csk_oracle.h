/*
 * csk_oracle.h -- plain CPU oracle for the Count Sketch Kaczmarz (CSK) method
 * (Zhang & Li, "A Count Sketch Kaczmarz Method For Solving Large
 * Overdetermined Linear Systems", arXiv 2004.02480).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists so that the tests, the
 * smoke check and the CPU-baseline leg of the benchmark can check the CUDA
 * library against a slow, obviously correct restatement of the paper.  The
 * product path never links, loads or calls it, and it shares no source,
 * header, table or helper with the CUDA library.
 *
 * Conventions: every index is 0-based (the paper's [m], [d] are 1-based);
 * matrices are row-major with a leading dimension; all floating-point work is
 * IEEE binary64 except the two functions whose name says f32 / bf16, which
 * exist only to reproduce an exact FP32 (or BF16) rounding sequence for
 * bit-level comparisons.
 *
 * Status codes returned by the iteration: 0 converged, 1 iteration cap
 * reached, -4 numerical failure (no non-zero row, or a NaN/Inf residual).
 */
#ifndef CSK_ORACLE_H
#define CSK_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* SplitMix64 output for counter value c (c >= 1) of the stream started at
 * `seed`: mix64(seed + c * 0x9E3779B97F4A7C15), Steele, Lea & Flood (2014).
 * Used as the counter-based source of the count sketch's randomness. */
uint64_t or_splitmix64_at(uint64_t seed, uint64_t c);

/* Count sketch map of Definition 1: for every row i in [0, m), h[i] in
 * [0, d) (uniform, multiply-shift range reduction of the high 32 bits of
 * u_i = or_splitmix64_at(seed, i + 1)) and sign[i] = +1 or -1 (bit 0 of u_i:
 * 0 -> +1, 1 -> -1).  h and sign may each be NULL. */
void or_count_sketch_map(uint64_t seed, int64_t m, int64_t d,
                         int32_t *h, int8_t *sign);

/* Textbook stable counting sort of the rows by bucket: cnt[j] = #{i: h[i]=j},
 * off[j] = sum_{t<j} cnt[t] (off has d+1 entries, off[d] = m), and perm lists
 * the rows in (h[i], i) order.  Any output may be NULL. */
void or_stable_count_sort(const int32_t *h, int64_t m, int64_t d,
                          int32_t *cnt, int32_t *off, int32_t *perm);

/* Sketch of Algorithm 1 (Initialize): At = S A (d x n, ld n) and
 * bt = S B (d x nrhs, ld nrhs) with S = Phi D from (h, sign).  Rows are added
 * in ascending original index.  B / bt may be NULL. */
void or_sketch_f64(const double *A, int64_t m, int64_t n, int64_t lda,
                   const double *B, int64_t ldb, int64_t nrhs,
                   const int32_t *h, const int8_t *sign, int64_t d,
                   double *At, double *bt);

/* The same sketch with FP32 inputs and FP32 sequential additions in
 * ascending original row index: the exact rounding sequence a fixed-order
 * FP32 implementation must reproduce bit for bit. */
void or_sketch_f32_same_order(const float *A, int64_t m, int64_t n,
                              int64_t lda, const float *B, int64_t ldb,
                              int64_t nrhs, const int32_t *h,
                              const int8_t *sign, int64_t d,
                              float *At, float *bt);

/* Squared row norms N[j] = ||At_j||_2^2 (binary64 accumulation, ascending
 * column order), for FP64 or FP32 At. */
void or_row_norms2_f64(const double *At, int64_t d, int64_t n, int64_t ld,
                       double *N);
void or_row_norms2_of_f32(const float *At, int64_t d, int64_t n, int64_t ld,
                          double *N);

/* Maximal-weighted-residual Kaczmarz loop of Algorithm 1 on (At, bt)
 * (d x n), run literally: each step recomputes the full residual
 * r = bt - At x, picks i_k = argmax |r_j| / ||At_j|| over rows with
 * ||At_j|| > 0 (ties -> smallest j) and projects x onto row i_k.
 *
 * Stopping (Section 3): with x_star != NULL the test RES = ||x-x*||^2/||x*||^2
 * <= tol is made before every step; with x_star == NULL the test is
 * ||bt - At x||^2 / ||bt||^2 <= tol.  The loop also stops when k reaches
 * max_iter (status 1) or when every weighted residual is exactly 0.
 * *iters receives the number of updates performed.
 *
 * nthreads > 1 computes the residual rows on that many OpenMP threads; each
 * row is still one sequential dot product, so the result does not depend on
 * the thread count.
 *
 * Optional per-step logs (length log_len, entry k for step k < log_len):
 *   ik_log[k]  = i_k
 *   gap_log[k] = (t1 - t2) / t1 for the two largest |r_j|/||At_j|| (0 if <2 rows)
 *   err2_log[k]= ||x_k - x*||^2 (needs x_star)
 *   rik_log[k] = r_{i_k}
 *   nik_log[k] = ||At_{i_k}||^2
 */
int or_mwrk(const double *At, const double *bt, int64_t d, int64_t n,
            int64_t ld, const double *x0, const double *x_star, double tol,
            int64_t max_iter, int nthreads, double *x, int64_t *iters,
            int64_t log_len, int32_t *ik_log, double *gap_log,
            double *err2_log, double *rik_log, double *nik_log);

/* Whole CSK method (Algorithm 1): sketch map from seed, sketch, then or_mwrk
 * on the sketch.  d == 0 selects MWRK on A itself (S = I, Remark 1). */
int or_csk(const double *A, const double *b, int64_t m, int64_t n,
           int64_t lda, int64_t d, uint64_t seed, const double *x0,
           const double *x_star, double tol, int64_t max_iter, int nthreads,
           double *x, int64_t *iters);

/* Final check quantities in binary64: *rse = ||x - x*||^2/||x*||^2 (if
 * x_star != NULL, else NaN) and *resid = ||bt - At x|| / ||bt||. */
void or_final_check(const double *At, const double *bt, int64_t d, int64_t n,
                    int64_t ld, const double *x, const double *x_star,
                    double *rse, double *resid);

/* Round-to-nearest-even conversion of a binary32 value to bfloat16, returned
 * as the binary32 value it represents. */
float or_bf16_round(float v);

/* Gram matrix G = At At^T (d x d) in binary64, and the split-BF16 product
 * that a tensor-core implementation forms: with hi = bf16(a), lo = bf16(a-hi),
 * G_ij = sum_c hi_ic hi_jc + hi_ic lo_jc + lo_ic hi_jc, summed in binary64.
 * G_ij is written for every (i, j). */
void or_gram_f64(const double *At, int64_t d, int64_t n, int64_t ld,
                 double *G);
void or_gram_split_bf16(const float *At, int64_t d, int64_t n, int64_t ld,
                        double *G);

/* Rows rows[0..nrows) of the split-BF16 product above (nrows x d, binary64),
 * for checks at sizes where the whole d x d matrix is too large. */
void or_gram_split_bf16_rows(const float *At, int64_t d, int64_t n, int64_t ld,
                             const int64_t *rows, int64_t nrows, double *Grows);

#ifdef __cplusplus
}
#endif

#endif
