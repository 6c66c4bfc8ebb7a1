/*
 * The oracle's CSR SpMV row loop run on every host core (OpenMP), for the
 * benchmark's all-cores CPU baseline.  TEST INFRASTRUCTURE ONLY, like
 * oracle.c: only the tests and the benchmark's CPU-baseline leg call it.
 *
 * Each row is the plain definition of y_i = alpha sum_k val_k x_{col_k} +
 * beta y_i (paper, Sec. 6.1), summed in column order with separate
 * multiply and add (compiled with -ffp-contract=off), exactly as
 * orc_spmv_csr in oracle.c does; rows are shared out among threads in
 * contiguous blocks, so the result is bit-identical to the single-thread
 * oracle.  Kept in its own file and library so that oracle.c stays a
 * plain sequential program.
 */
#include <stdint.h>

void orc_spmv_csr_omp(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
                      const double *x, double alpha, double beta, double *y, int threads)
{
#pragma omp parallel for schedule(static) num_threads(threads)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            double p = val[k] * x[col[k]];
            s = s + p;
        }
        double out = alpha * s;
        if (beta != 0.0) {
            double t = beta * y[i];
            out = out + t;
        }
        y[i] = out;
    }
}
