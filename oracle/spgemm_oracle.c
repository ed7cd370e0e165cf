/*
 * CPU oracle for CSR sparse matrix-matrix multiplication C = A*B.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or
 * calls this file; it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA library against a plain,
 * slow, obviously correct implementation.  It shares no code, header or
 * table with the CUDA library.
 *
 * Method followed: the row-wise (Gustavson) formulation of Section 2.1 of
 * Deveci et al., "Sparse Matrix-Matrix Multiplication on Multilevel Memory
 * Architectures": row i of C is the sum over the stored entries a_ik of row i
 * of A of a_ik times row k of B, with rows of A processed one after another
 * and each row of B read through in stored order (Section 2.1, Figure 1).
 * The symbolic phase counts the distinct columns of each row of C and the
 * numeric phase produces the values (the two phases of Section 2.1).
 *
 * The accumulator is the dense accumulator that Section 3.1 contrasts with
 * the hashmap accumulator: a value array and a marker array as long as the
 * number of columns of B.  All arithmetic is in IEEE double precision;
 * single-precision inputs are promoted by the caller before the call.
 *
 * Readings of the paper that this file takes (the paper is silent on them):
 *  - the output pattern is structural: an entry (i,j) exists when some stored
 *    a_ik and stored b_kj meet, even if the sum is exactly zero;
 *  - columns of each output row are emitted in ascending order;
 *  - input columns may be unsorted within a row (Section 3.2.2 states that the
 *    kernel does not assume sorted columns); a duplicate column inside one
 *    input row is an input error (see oracle_validate_csr);
 *  - c_bound[p] = sum over contributing terms of |a_ik|*|b_kj| is returned
 *    with each value so that a tolerance can be stated per entry.
 *
 * Rows [r0, r1) of A are processed; outputs are written relative to r0.
 * OpenMP distributes rows over threads; every thread owns its accumulator.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Returns 0 if the CSR arrays are well formed, 1 if row_ptr is not
 * non-decreasing or does not start at 0, 2 if a column is out of range,
 * 3 if a row holds the same column twice. */
int oracle_validate_csr(int64_t nrows, int64_t ncols, const int64_t *rp,
                        const int32_t *col) {
    if (rp[0] != 0) return 1;
    for (int64_t i = 0; i < nrows; i++)
        if (rp[i + 1] < rp[i]) return 1;
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncols > 0 ? ncols : 1));
    if (!mark) return -1;
    for (int64_t j = 0; j < ncols; j++) mark[j] = -1;
    int rc = 0;
    for (int64_t i = 0; i < nrows && rc == 0; i++) {
        for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
            int64_t j = col[p];
            if (j < 0 || j >= ncols) { rc = 2; break; }
            if (mark[j] == i) { rc = 3; break; }
            mark[j] = i;
        }
    }
    free(mark);
    return rc;
}

/* Symbolic phase: cnt[i-r0] = number of distinct columns of row i of C,
 * mults[i-r0] = number of products a_ik*b_kj that row i takes
 * (Section 3.1: the number of accumulator insertions equals the number of
 * multiplications).  Returns 0, or -1 on allocation failure. */
int oracle_symbolic_rows(int64_t r0, int64_t r1, int64_t ncols_b,
                         const int64_t *a_rp, const int32_t *a_col,
                         const int64_t *b_rp, const int32_t *b_col,
                         int64_t *cnt, int64_t *mults) {
    int fail = 0;
#pragma omp parallel
    {
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncols_b > 0 ? ncols_b : 1));
        if (!mark) {
#pragma omp atomic write
            fail = 1;
        } else {
            for (int64_t j = 0; j < ncols_b; j++) mark[j] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = r0; i < r1; i++) {
                int64_t c = 0, m = 0;
                for (int64_t p = a_rp[i]; p < a_rp[i + 1]; p++) {
                    int64_t k = a_col[p];
                    for (int64_t q = b_rp[k]; q < b_rp[k + 1]; q++) {
                        int64_t j = b_col[q];
                        m++;
                        if (mark[j] != i) { mark[j] = i; c++; }
                    }
                }
                cnt[i - r0] = c;
                if (mults) mults[i - r0] = m;
            }
            free(mark);
        }
    }
    return fail ? -1 : 0;
}

static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* Numeric phase for rows [r0, r1).  c_rp holds r1-r0+1 offsets relative to
 * the first output row (c_rp[0] == 0), as produced from the symbolic counts.
 * For every row: walk the stored entries of A's row in stored order, walk the
 * matching row of B in stored order, accumulate a_ik*b_kj into acc[j]
 * (Section 2.1), then emit the touched columns in ascending order.
 * c_bound may be NULL.  Returns 0, -1 on allocation failure, -2 if a row's
 * distinct column count disagrees with c_rp. */
int oracle_numeric_rows(int64_t r0, int64_t r1, int64_t ncols_b,
                        const int64_t *a_rp, const int32_t *a_col, const double *a_val,
                        const int64_t *b_rp, const int32_t *b_col, const double *b_val,
                        const int64_t *c_rp, int32_t *c_col, double *c_val,
                        double *c_bound) {
    int fail = 0;
#pragma omp parallel
    {
        size_t nc = (size_t)(ncols_b > 0 ? ncols_b : 1);
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * nc);
        double *acc = (double *)malloc(sizeof(double) * nc);
        double *bnd = (double *)malloc(sizeof(double) * nc);
        if (!mark || !acc || !bnd) {
#pragma omp atomic write
            fail = -1;
        } else {
            for (size_t j = 0; j < nc; j++) mark[j] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = r0; i < r1; i++) {
                int64_t out = c_rp[i - r0], cap = c_rp[i - r0 + 1];
                int64_t w = out;
                int ok = 1;
                for (int64_t p = a_rp[i]; p < a_rp[i + 1]; p++) {
                    int64_t k = a_col[p];
                    double a = a_val[p];
                    for (int64_t q = b_rp[k]; q < b_rp[k + 1]; q++) {
                        int64_t j = b_col[q];
                        double prod = a * b_val[q];
                        if (mark[j] != i) {
                            mark[j] = i;
                            acc[j] = 0.0;
                            bnd[j] = 0.0;
                            if (w < cap) c_col[w] = (int32_t)j;
                            w++;
                        }
                        acc[j] += prod;
                        bnd[j] += fabs(a) * fabs(b_val[q]);
                    }
                }
                if (w != cap) ok = 0;
                if (ok) {
                    qsort(c_col + out, (size_t)(cap - out), sizeof(int32_t), cmp_i32);
                    for (int64_t t = out; t < cap; t++) {
                        c_val[t] = acc[c_col[t]];
                        if (c_bound) c_bound[t] = bnd[c_col[t]];
                    }
                } else {
#pragma omp atomic write
                    fail = -2;
                }
            }
        }
        free(mark); free(acc); free(bnd);
    }
    return fail;
}

/* Row-range fused multiply-add of Section 3.2.2 (the subprocedure used by the
 * chunking methods, Algorithms 1-3): for rows [r0, r1) of A,
 *     C2_i = sum over stored a_ik with lo <= k < hi of a_ik * B_k  +  C1_i,
 * where C1 is a partial result in compact CSR (p_rp relative to r0, columns
 * in any order).  Columns of A outside [lo, hi) are skipped, not assumed
 * sorted.  Called twice: first with o_col == NULL to fill o_cnt (distinct
 * columns per row), then with o_rp (relative offsets) to fill columns (sorted)
 * and values.  Returns 0 or -1 on allocation failure. */
int oracle_fma_range_rows(int64_t r0, int64_t r1, int64_t ncols_b, int64_t lo, int64_t hi,
                          const int64_t *a_rp, const int32_t *a_col, const double *a_val,
                          const int64_t *b_rp, const int32_t *b_col, const double *b_val,
                          const int64_t *p_rp, const int32_t *p_col, const double *p_val,
                          int64_t *o_cnt, const int64_t *o_rp, int32_t *o_col, double *o_val) {
    int fail = 0;
#pragma omp parallel
    {
        size_t nc = (size_t)(ncols_b > 0 ? ncols_b : 1);
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * nc);
        double *acc = (double *)malloc(sizeof(double) * nc);
        int32_t *list = (int32_t *)malloc(sizeof(int32_t) * nc);
        if (!mark || !acc || !list) {
#pragma omp atomic write
            fail = -1;
        } else {
            for (size_t j = 0; j < nc; j++) mark[j] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = r0; i < r1; i++) {
                int64_t n = 0;
                for (int64_t p = a_rp[i]; p < a_rp[i + 1]; p++) {
                    int64_t k = a_col[p];
                    if (k < lo || k >= hi) continue;
                    double a = a_val ? a_val[p] : 0.0;
                    for (int64_t q = b_rp[k]; q < b_rp[k + 1]; q++) {
                        int64_t j = b_col[q];
                        if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; list[n++] = (int32_t)j; }
                        if (o_col) acc[j] += a * b_val[q];
                    }
                }
                if (p_rp) {
                    for (int64_t t = p_rp[i - r0]; t < p_rp[i - r0 + 1]; t++) {
                        int64_t j = p_col[t];
                        if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; list[n++] = (int32_t)j; }
                        if (o_col) acc[j] += p_val[t];
                    }
                }
                if (!o_col) {
                    o_cnt[i - r0] = n;
                } else {
                    qsort(list, (size_t)n, sizeof(int32_t), cmp_i32);
                    int64_t base = o_rp[i - r0];
                    for (int64_t t = 0; t < n; t++) {
                        o_col[base + t] = list[t];
                        o_val[base + t] = acc[list[t]];
                    }
                }
            }
        }
        free(mark); free(acc); free(list);
    }
    return fail;
}

/* Gradients of L(A,B) = <dC, A*B> restricted to the stored patterns of A and
 * B (the product is bilinear, so these are the exact partial derivatives):
 *     dA_ik = sum over stored b_kj of dC_ij * b_kj,
 *     dB_kj = sum over stored a_ik of a_ik * dC_ij,
 * where dC is given on the pattern of C (c_rp, c_col: every (i,j) reached by
 * the product must be present).  Rows are walked in order; no parallelism,
 * so dB accumulates without races.  Returns 0, -1 on allocation failure,
 * -2 if a product entry is missing from C's pattern. */
int oracle_backward(int64_t n_a, int64_t ncols_b,
                    const int64_t *a_rp, const int32_t *a_col, const double *a_val,
                    const int64_t *b_rp, const int32_t *b_col, const double *b_val,
                    const int64_t *c_rp, const int32_t *c_col, const double *dc_val,
                    double *da, double *db) {
    size_t nc = (size_t)(ncols_b > 0 ? ncols_b : 1);
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * nc);
    double *dense = (double *)malloc(sizeof(double) * nc);
    if (!mark || !dense) { free(mark); free(dense); return -1; }
    for (size_t j = 0; j < nc; j++) mark[j] = -1;
    /* dB is accumulated into: the caller passes a zeroed array. */
    int rc = 0;
    for (int64_t i = 0; i < n_a && rc == 0; i++) {
        for (int64_t t = c_rp[i]; t < c_rp[i + 1]; t++) {
            mark[c_col[t]] = i;
            dense[c_col[t]] = dc_val[t];
        }
        for (int64_t p = a_rp[i]; p < a_rp[i + 1]; p++) {
            int64_t k = a_col[p];
            double g = 0.0;
            for (int64_t q = b_rp[k]; q < b_rp[k + 1]; q++) {
                int64_t j = b_col[q];
                if (mark[j] != i) { rc = -2; break; }
                g += dense[j] * b_val[q];
                if (db) db[q] += a_val[p] * dense[j];
            }
            if (da) da[p] = g;
        }
    }
    free(mark); free(dense);
    return rc;
}
