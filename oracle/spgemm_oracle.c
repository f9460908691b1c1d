/*
 * CPU oracle for row-wise (Gustavson) SpGEMM, C = A * B.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library. The CUDA library
 * shares no code, header or helper with it.
 *
 * Everything here is written from the definitions of the method, not from
 * any GPU design:
 *   - the product (Eq. 1, Eq. 2): C_i* = sum over k in A_i* of A_ik * B_k*;
 *   - the CSR layout (Sec. 2.1.1): rpt (M+1), col and val, columns ascending
 *     and unique inside each output row;
 *   - the intermediate-product count n_prod of a row (Sec. 2.1.2, Eq. 3):
 *     the number of (A entry, B entry) pairs that meet in that row;
 *   - the symbolic phase (Sec. 2.2, Algorithm 4): n_nz of a row is the number
 *     of distinct column keys among those products. Products whose sum
 *     cancels to 0.0 stay in the structure, because the symbolic phase counts
 *     keys, not values;
 *   - the numeric phase (Sec. 2.2, Algorithm 5): the values of products that
 *     share a key are summed.
 * The accumulator is a dense array indexed by column with a "last row seen"
 * marker (a textbook Gustavson dense accumulator), which is obviously exact
 * and needs no hashing. Products are summed in stored order: for each A
 * entry in stored order, for each B entry of row k in stored order, with
 * plain IEEE double multiply and add (built with -ffp-contract=off so no FMA
 * is fused in).
 *
 * Index conventions: row pointers are int64, column indices int32, values
 * double. Functions return 0 on success, a negative code on bad input
 * (-1 out-of-range column, -2 non-monotone row pointer, -3 out of memory).
 */
#include <stdint.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int check_csr(int64_t rows, int64_t cols, const int64_t *rpt,
                     const int32_t *col)
{
    if (rpt[0] != 0) return -2;
    for (int64_t i = 0; i < rows; ++i) {
        if (rpt[i + 1] < rpt[i]) return -2;
        for (int64_t p = rpt[i]; p < rpt[i + 1]; ++p)
            if (col[p] < 0 || (int64_t)col[p] >= cols) return -1;
    }
    return 0;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Setup step (Sec. 5, step 1): n_prod[i] = sum over A entries (i,k) of the
 * length of row k of B. */
int oracle_nprod(int64_t M, int64_t K, const int64_t *arpt, const int32_t *acol,
                 const int64_t *brpt, int64_t *nprod)
{
    int rc = check_csr(M, K, arpt, acol);
    if (rc) return rc;
    for (int64_t i = 0; i < M; ++i) {
        int64_t s = 0;
        for (int64_t p = arpt[i]; p < arpt[i + 1]; ++p) {
            int64_t k = acol[p];
            s += brpt[k + 1] - brpt[k];
        }
        nprod[i] = s;
    }
    return 0;
}

/* Symbolic phase (Sec. 2.2, Algorithm 4): for rows [r0, r1) count the
 * distinct column keys of the products. nnz[i - r0] receives the count. */
int oracle_symbolic(int64_t r0, int64_t r1, int64_t K, int64_t N,
                    const int64_t *arpt, const int32_t *acol,
                    const int64_t *brpt, const int32_t *bcol,
                    int64_t *nnz, int nthreads)
{
    int rc = 0;
    set_threads(nthreads);
#pragma omp parallel
    {
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
        if (!mark) {
#pragma omp atomic write
            rc = -3;
        } else {
            for (int64_t j = 0; j < N; ++j) mark[j] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = r0; i < r1; ++i) {
                int64_t count = 0;
                for (int64_t p = arpt[i]; p < arpt[i + 1]; ++p) {
                    int64_t k = acol[p];
                    for (int64_t q = brpt[k]; q < brpt[k + 1]; ++q) {
                        int32_t j = bcol[q];
                        if (mark[j] != i) { mark[j] = i; ++count; }
                    }
                }
                nnz[i - r0] = count;
            }
            free(mark);
        }
    }
    (void)K;
    return rc;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Numeric phase (Sec. 2.2, Algorithm 5) plus the output layout of
 * Sec. 2.1.1: for rows [r0, r1) write the sorted unique columns and summed
 * values at crpt[i - r0] .. crpt[i - r0 + 1] (crpt relative to the window,
 * as produced by an exclusive scan of the symbolic counts). cabs, if not
 * NULL, receives sum |a_ik * b_kj| per entry: the scale of the rounding
 * error bound used by the value tolerance. */
int oracle_numeric(int64_t r0, int64_t r1, int64_t K, int64_t N,
                   const int64_t *arpt, const int32_t *acol, const double *aval,
                   const int64_t *brpt, const int32_t *bcol, const double *bval,
                   const int64_t *crpt, int32_t *ccol, double *cval, double *cabs,
                   int nthreads)
{
    int rc = 0;
    set_threads(nthreads);
#pragma omp parallel
    {
        size_t n1 = (size_t)(N > 0 ? N : 1);
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * n1);
        double *acc = (double *)malloc(sizeof(double) * n1);
        double *aab = (double *)malloc(sizeof(double) * n1);
        int32_t *list = (int32_t *)malloc(sizeof(int32_t) * n1);
        if (!mark || !acc || !aab || !list) {
#pragma omp atomic write
            rc = -3;
        } else {
            for (int64_t j = 0; j < N; ++j) mark[j] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = r0; i < r1; ++i) {
                int64_t len = 0;
                for (int64_t p = arpt[i]; p < arpt[i + 1]; ++p) {
                    int64_t k = acol[p];
                    double a = aval[p];
                    for (int64_t q = brpt[k]; q < brpt[k + 1]; ++q) {
                        int32_t j = bcol[q];
                        double prod = a * bval[q];
                        if (mark[j] != i) {
                            mark[j] = i;
                            acc[j] = 0.0;
                            aab[j] = 0.0;
                            list[len++] = j;
                        }
                        acc[j] = acc[j] + prod;
                        aab[j] = aab[j] + (prod < 0 ? -prod : prod);
                    }
                }
                qsort(list, (size_t)len, sizeof(int32_t), cmp_i32);
                int64_t base = crpt[i - r0];
                if (crpt[i - r0 + 1] - base != len) {
#pragma omp atomic write
                    rc = -4;
                    continue;
                }
                for (int64_t t = 0; t < len; ++t) {
                    ccol[base + t] = list[t];
                    cval[base + t] = acc[list[t]];
                    if (cabs) cabs[base + t] = aab[list[t]];
                }
            }
        }
        free(mark); free(acc); free(aab); free(list);
    }
    (void)K;
    return rc;
}

/* Order-free summary of rows [r0, r1) for checks at sizes where all of C
 * cannot be held on the host: per row the entry count, the sum of column
 * indices and the sum of values (summed in column order, so the sum is the
 * same for any correct C). */
int oracle_row_checksums(int64_t r0, int64_t r1, int64_t K, int64_t N,
                         const int64_t *arpt, const int32_t *acol, const double *aval,
                         const int64_t *brpt, const int32_t *bcol, const double *bval,
                         int64_t *cnt, int64_t *colsum, double *valsum, double *abssum,
                         int nthreads)
{
    int rc = 0;
    set_threads(nthreads);
#pragma omp parallel
    {
        size_t n1 = (size_t)(N > 0 ? N : 1);
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * n1);
        double *acc = (double *)malloc(sizeof(double) * n1);
        int32_t *list = (int32_t *)malloc(sizeof(int32_t) * n1);
        if (!mark || !acc || !list) {
#pragma omp atomic write
            rc = -3;
        } else {
            for (int64_t j = 0; j < N; ++j) mark[j] = -1;
#pragma omp for schedule(dynamic, 16)
            for (int64_t i = r0; i < r1; ++i) {
                int64_t len = 0;
                double as = 0.0;   /* sum over the row's products of |a*b| */
                for (int64_t p = arpt[i]; p < arpt[i + 1]; ++p) {
                    int64_t k = acol[p];
                    double a = aval[p];
                    for (int64_t q = brpt[k]; q < brpt[k + 1]; ++q) {
                        int32_t j = bcol[q];
                        if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; list[len++] = j; }
                        acc[j] = acc[j] + a * bval[q];
                        as = as + fabs(a * bval[q]);
                    }
                }
                qsort(list, (size_t)len, sizeof(int32_t), cmp_i32);
                int64_t cs = 0;
                double vs = 0.0;
                for (int64_t t = 0; t < len; ++t) { cs += list[t]; vs += acc[list[t]]; }
                cnt[i - r0] = len;
                colsum[i - r0] = cs;
                valsum[i - r0] = vs;
                if (abssum) abssum[i - r0] = as;
            }
        }
        free(mark); free(acc); free(list);
    }
    (void)K;
    return rc;
}

int oracle_check_csr(int64_t rows, int64_t cols, const int64_t *rpt, const int32_t *col)
{
    return check_csr(rows, cols, rpt, col);
}
