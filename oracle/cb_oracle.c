/*
 * CPU oracle for the blocked SpMV -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load this library. The product path (the CUDA library and its Python binding) never
 * calls it and shares no code with it.
 *
 * What it computes is the plain definition of the sparse matrix-vector product the
 * paper accelerates: the row-parallel CSR SpMV of Sec. 2.2, Algorithm 1,
 *     y_i = sum_{k=row_ptr[i]}^{row_ptr[i+1]-1} val[k] * x[col[k]],
 * extended with the BLAS scaling y <- alpha*A*x + beta*y (beta == 0 means y is not read).
 * Sums run sequentially in CSR order in IEEE double; the file is compiled with
 * -ffp-contract=off so every product is rounded before it is added.
 *
 * Besides y it returns, per row, s_i = sum_k |val[k] * x[col[k]]|, the scale that the
 * acceptance test divides the error by.
 *
 * A brute-force dense product in long double serves as an independent check on tiny
 * inputs.
 *
 * ORACLE_MUTANT (compile-time, tests only) plants a known mistake so that the test
 * suite can show that its pins catch it:
 *   1 drops the last entry of every row, 2 reads x at the previous entry's column,
 *   3 swaps the roles of alpha and beta, 4 adds beta*y even when beta == 0,
 *   5 transposes (scatters A^T x instead of gathering A x).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

static void row_product(const int64_t* row_ptr, const int32_t* col, const double* val,
                        const double* x, int64_t i, double* sum_out, double* abs_out) {
  double sum = 0.0, sabs = 0.0;
  int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
#if ORACLE_MUTANT == 1
  if (hi > lo) hi -= 1;
#endif
  for (int64_t k = lo; k < hi; ++k) {
    int64_t c = col[k];
#if ORACLE_MUTANT == 2
    if (k > lo) c = col[k - 1];
#endif
    double p = val[k] * x[c];
    sum = sum + p;
    sabs = sabs + fabs(p);
  }
  *sum_out = sum;
  *abs_out = sabs;
}

static double finish(double alpha, double beta, double sum, const double* y0, int64_t i) {
#if ORACLE_MUTANT == 3
  { double t = alpha; alpha = beta; beta = t; }
  return alpha * sum + beta * (y0 ? y0[i] : 0.0);
#elif ORACLE_MUTANT == 4
  return alpha * sum + beta * (y0 ? y0[i] : 0.0);
#else
  if (beta == 0.0) return alpha * sum;
  return alpha * sum + beta * y0[i];
#endif
}

/* y[i] = alpha * (A x)_i + beta * y0[i] for all rows; s[i] = sum |a_ik x_k| (s may be NULL).
 * y0 may equal y (in-place) and is not read when beta == 0. */
void oracle_spmv_csr(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                     const double* x, double alpha, double beta, const double* y0, double* y,
                     double* s) {
#if ORACLE_MUTANT == 5
  for (int64_t i = 0; i < m; ++i) {
    double yi = (beta == 0.0) ? 0.0 : beta * y0[i];
    y[i] = yi;
    if (s) s[i] = 0.0;
  }
  for (int64_t i = 0; i < m; ++i)
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      int64_t c = col[k];
      if (c < m && i < n) {            /* stays inside y and x for any shape */
        y[c] += alpha * val[k] * x[i];
        if (s) s[c] += fabs(val[k] * x[i]);
      }
    }
#else
  for (int64_t i = 0; i < m; ++i) {
    double sum, sabs;
    row_product(row_ptr, col, val, x, i, &sum, &sabs);
    y[i] = finish(alpha, beta, sum, y0, i);
    if (s) s[i] = sabs;
  }
#endif
}

/* The same product for a list of rows only (used to check sampled rows of large
 * matrices): y[j], s[j] refer to row rows[j]; y0 is indexed by row. */
void oracle_spmv_csr_rows(int64_t nrows, const int64_t* rows, const int64_t* row_ptr,
                          const int32_t* col, const double* val, const double* x, double alpha,
                          double beta, const double* y0, double* y, double* s) {
  for (int64_t j = 0; j < nrows; ++j) {
    int64_t i = rows[j];
    double sum, sabs;
    row_product(row_ptr, col, val, x, i, &sum, &sabs);
    y[j] = finish(alpha, beta, sum, y0, i);
    if (s) s[j] = sabs;
  }
}

/* k right-hand sides: X is k x n row-major (ldx >= n), Y and Y0 are k x m (ldy >= m). */
void oracle_spmm_csr(int64_t m, int64_t k, const int64_t* row_ptr, const int32_t* col,
                     const double* val, const double* X, int64_t ldx, double alpha, double beta,
                     const double* Y0, int64_t ldy, double* Y, double* S) {
  for (int64_t j = 0; j < k; ++j)
    oracle_spmv_csr(m, ldx, row_ptr, col, val, X + j * ldx, alpha, beta,
                    Y0 ? Y0 + j * ldy : (const double*)0, Y + j * ldy, S ? S + j * ldy : 0);
}

/* Dense brute force in long double: y[i] = sum_j A[i*n + j] * x[j] (A row-major). */
void oracle_dense_gemv_ld(int64_t m, int64_t n, const double* A, const double* x, double* y) {
  for (int64_t i = 0; i < m; ++i) {
    long double acc = 0.0L;
    for (int64_t j = 0; j < n; ++j) acc += (long double)A[i * n + j] * (long double)x[j];
    y[i] = (double)acc;
  }
}

int oracle_mutant_id(void) { return ORACLE_MUTANT; }
