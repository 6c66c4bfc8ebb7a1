/*
 * Plain FP64 CPU oracle for the sparse hot path: SpMV in every storage
 * format, the format conversions, conjugate gradients (plain, mixed-precision
 * with iterative refinement, batched), dense Cholesky, compensated dot
 * products and the matrix statistics of the format selector.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call
 * this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA library.
 *
 * Every routine follows the plain definition of what it computes, with
 * loops in the order of that definition and no blocking, fusion or
 * reordering.  Floating-point multiply and add are separate operations:
 * the file is compiled with -ffp-contract=off so that no multiply-add is
 * fused and results are identical on every host.
 *
 * Sources: the paper (Cojean, Tsai, Anzt, "Ginkgo - A Math Library designed
 * for Platform Portability", Sec. 6.1 for SpMV and its COO/CSR byte bounds,
 * Sec. 6.2 for Krylov solvers built on SpMV); the formats it refers to but
 * does not define follow their standard definitions: ELL and hybrid ELL+COO
 * (Bell and Garland, SC'09), SELL-P (Anzt, Tomov and Dongarra, 2014);
 * CG is the method of Hestenes and Stiefel (1952), also in the
 * single-reduction form of Chronopoulos and Gear (1989) and preconditioned by
 * the diagonal (Jacobi); BiCGSTAB is van der Vorst's (1992), GMRES Saad and
 * Schultz's (1986); Dot2 is Algorithm 5.3 of
 * Ogita, Rump and Oishi, "Accurate sum and dot product" (SISC 2005).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_CONVERGED 6
#define ORC_BREAKDOWN 7
#define ORC_INVALID 1

/* ------------------------------------------------------------------ SpMV */

/* y_i = alpha * sum_k val_k x_{col_k} + beta * y_i over the stored entries
 * k of row i in ascending position (= ascending column) order.  beta == 0
 * means y is not read (BLAS convention), so NaN in y does not propagate.
 * Sec. 6.1: the product y = A x of a CSR matrix. */
void orc_spmv_csr(int64_t n, const int32_t *row_ptr, const int32_t *col,
                  const double *val, const double *x, double alpha, double beta,
                  double *y)
{
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

/* Error-free transformations (Ogita-Rump-Oishi 2005, Algorithms 3.1, 3.3):
 * TwoSum gives s + e = a + b exactly; TwoProduct gives p + e = a * b
 * exactly, with the error term taken from the correctly rounded C99 fma(). */
static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double z = x - a;
    double t1 = a - (x - z);
    double t2 = b - z;
    *s = x;
    *e = t1 + t2;
}

static void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

/* Near-exact reference of orc_spmv_csr with Dot2 (compensated dot product,
 * result as accurate as if computed in twice the working precision), plus
 * the magnitude mag_i = |alpha| sum_k |val_k x_{col_k}| + |beta| |y_i| that
 * scales the per-entry tolerance.  y_in may be NULL when beta == 0. */
void orc_spmv_csr_dot2(int64_t n, const int32_t *row_ptr, const int32_t *col,
                       const double *val, const double *x, double alpha, double beta,
                       const double *y_in, double *y_out, double *mag)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0, c = 0.0, m = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            double p, e1, e2;
            two_prod(val[k], x[col[k]], &p, &e1);
            two_sum(s, p, &s, &e2);
            c = c + (e1 + e2);
            m = m + fabs(val[k] * x[col[k]]);
        }
        /* alpha * (s + c) and beta * y, again compensated */
        double r = 0.0, rc = 0.0, p, e1, e2;
        two_prod(alpha, s, &p, &e1);
        two_sum(r, p, &r, &e2);
        rc = rc + e1 + e2 + alpha * c;
        double mm = fabs(alpha) * m;
        if (beta != 0.0) {
            two_prod(beta, y_in[i], &p, &e1);
            two_sum(r, p, &r, &e2);
            rc = rc + e1 + e2;
            mm = mm + fabs(beta) * fabs(y_in[i]);
        }
        y_out[i] = r + rc;
        if (mag)
            mag[i] = mm;
    }
}

/* COO: entries (row_k, col_k, val_k) in (row, col) order; each row's sum
 * is formed over its entries in that order.  Sec. 6.1 (COO format). */
void orc_spmv_coo(int64_t n, int64_t nnz, const int32_t *row, const int32_t *col,
                  const double *val, const double *x, double alpha, double beta,
                  double *y)
{
    double *s = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int64_t k = 0; k < nnz; ++k) {
        double p = val[k] * x[col[k]];
        s[row[k]] = s[row[k]] + p;
    }
    for (int64_t i = 0; i < n; ++i) {
        double out = alpha * s[i];
        if (beta != 0.0) {
            double t = beta * y[i];
            out = out + t;
        }
        y[i] = out;
    }
    free(s);
}

/* ELL: K slots per row, column-major with leading dimension n_pad:
 * slot (i, k) is at k * n_pad + i; a padding slot has col == -1 and is
 * skipped.  (Bell and Garland 2009.) */
void orc_spmv_ell(int64_t n, int64_t n_pad, int64_t K, const int32_t *col,
                  const double *val, const double *x, double alpha, double beta,
                  double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            int32_t c = col[k * n_pad + i];
            if (c < 0)
                continue;
            double p = val[k * n_pad + i] * x[c];
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

/* SELL-P: rows in slices of S; slice s has width slice_len[s] and starts at
 * column offset slice_set[s] (in units of S-slot columns); row r = s*S + l,
 * slot k of the row is at (slice_set[s] + k) * S + l.  Padding col == -1.
 * (Anzt, Tomov, Dongarra 2014.) */
void orc_spmv_sellp(int64_t n, int64_t S, const int32_t *slice_len,
                    const int32_t *slice_set, const int32_t *col, const double *val,
                    const double *x, double alpha, double beta, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t s_id = i / S, l = i % S;
        double s = 0.0;
        for (int64_t k = 0; k < slice_len[s_id]; ++k) {
            int64_t slot = ((int64_t)slice_set[s_id] + k) * S + l;
            int32_t c = col[slot];
            if (c < 0)
                continue;
            double p = val[slot] * x[c];
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

/* Hybrid ELL + COO: row i's sum is its ELL slots (in slot order) followed
 * by its COO entries (in order), i.e. its entries in column order. */
void orc_spmv_hybrid(int64_t n, int64_t n_pad, int64_t K, const int32_t *ell_col,
                     const double *ell_val, int64_t coo_nnz, const int32_t *coo_row,
                     const int32_t *coo_col, const double *coo_val, const double *x,
                     double alpha, double beta, double *y)
{
    double *s = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = 0; k < K; ++k) {
            int32_t c = ell_col[k * n_pad + i];
            if (c < 0)
                continue;
            double p = ell_val[k * n_pad + i] * x[c];
            s[i] = s[i] + p;
        }
    for (int64_t k = 0; k < coo_nnz; ++k) {
        double p = coo_val[k] * x[coo_col[k]];
        s[coo_row[k]] = s[coo_row[k]] + p;
    }
    for (int64_t i = 0; i < n; ++i) {
        double out = alpha * s[i];
        if (beta != 0.0) {
            double t = beta * y[i];
            out = out + t;
        }
        y[i] = out;
    }
    free(s);
}

/* ----------------------------------------------------------- conversions */

/* CSR -> COO: row index of every entry, entries in CSR order. */
void orc_csr_to_coo(int64_t n, const int32_t *row_ptr, const int32_t *col,
                    const double *val, int32_t *row_out, int32_t *col_out,
                    double *val_out)
{
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            row_out[k] = (int32_t)i;
            col_out[k] = col[k];
            val_out[k] = val[k];
        }
}

/* COO (sorted by row) -> CSR: row_ptr by counting entries per row. */
void orc_coo_to_csr(int64_t n, int64_t nnz, const int32_t *row, const int32_t *col,
                    const double *val, int32_t *row_ptr, int32_t *col_out,
                    double *val_out)
{
    for (int64_t i = 0; i <= n; ++i)
        row_ptr[i] = 0;
    for (int64_t k = 0; k < nnz; ++k)
        row_ptr[row[k] + 1] += 1;
    for (int64_t i = 0; i < n; ++i)
        row_ptr[i + 1] += row_ptr[i];
    for (int64_t k = 0; k < nnz; ++k) {
        col_out[k] = col[k];
        val_out[k] = val[k];
    }
}

/* Maximum row length. */
int64_t orc_max_row_len(int64_t n, const int32_t *row_ptr)
{
    int64_t K = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t L = row_ptr[i + 1] - row_ptr[i];
        if (L > K)
            K = L;
    }
    return K;
}

/* n rounded up to a multiple of 32: the ELL leading dimension. */
int64_t orc_ell_n_pad(int64_t n) { return (n + 31) / 32 * 32; }

/* CSR -> ELL of width K (K >= max row length): row i's entries fill its
 * first slots in column order, the rest are padding (col -1, val +0.0). */
void orc_csr_to_ell(int64_t n, int64_t n_pad, int64_t K, const int32_t *row_ptr,
                    const int32_t *col, const double *val, int32_t *ell_col,
                    double *ell_val)
{
    for (int64_t k = 0; k < K; ++k)
        for (int64_t i = 0; i < n_pad; ++i) {
            ell_col[k * n_pad + i] = -1;
            ell_val[k * n_pad + i] = 0.0;
        }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t slot = (k - row_ptr[i]) * n_pad + i;
            ell_col[slot] = col[k];
            ell_val[slot] = val[k];
        }
}

/* ELL -> CSR: drop padding slots (col == -1), keep slot order.  row_ptr
 * must have n+1 entries; col_out/val_out room for all non-padding slots. */
void orc_ell_to_csr(int64_t n, int64_t n_pad, int64_t K, const int32_t *ell_col,
                    const double *ell_val, int32_t *row_ptr, int32_t *col_out,
                    double *val_out)
{
    int64_t nz = 0;
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = 0; k < K; ++k) {
            int64_t slot = k * n_pad + i;
            if (ell_col[slot] < 0)
                continue;
            col_out[nz] = ell_col[slot];
            val_out[nz] = ell_val[slot];
            ++nz;
        }
        row_ptr[i + 1] = (int32_t)nz;
    }
}

/* SELL-P sizes: slice s (rows s*S .. s*S+S-1, clipped to n) has width
 * slice_len[s] = max row length in the slice rounded up to a multiple of the
 * stride factor f; slice_set is the exclusive prefix sum of the widths
 * (n_slices + 1 entries).  Returns the total number of slots
 * slice_set[n_slices] * S. */
int64_t orc_sellp_sizes(int64_t n, const int32_t *row_ptr, int64_t S, int64_t f,
                        int32_t *slice_len, int32_t *slice_set)
{
    int64_t n_slices = (n + S - 1) / S;
    int64_t acc = 0;
    for (int64_t s = 0; s < n_slices; ++s) {
        int64_t w = 0;
        for (int64_t i = s * S; i < (s + 1) * S && i < n; ++i) {
            int64_t L = row_ptr[i + 1] - row_ptr[i];
            if (L > w)
                w = L;
        }
        w = (w + f - 1) / f * f;
        slice_len[s] = (int32_t)w;
        slice_set[s] = (int32_t)acc;
        acc += w;
    }
    slice_set[n_slices] = (int32_t)acc;
    return acc * S;
}

/* CSR -> SELL-P with the sizes of orc_sellp_sizes. */
void orc_csr_to_sellp(int64_t n, int64_t S, const int32_t *row_ptr, const int32_t *col,
                      const double *val, const int32_t *slice_len,
                      const int32_t *slice_set, int32_t *s_col, double *s_val)
{
    int64_t n_slices = (n + S - 1) / S;
    int64_t total = (int64_t)slice_set[n_slices] * S;
    (void)slice_len; /* widths are implied by slice_set */
    for (int64_t t = 0; t < total; ++t) {
        s_col[t] = -1;
        s_val[t] = 0.0;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t s_id = i / S, l = i % S;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t slot = ((int64_t)slice_set[s_id] + (k - row_ptr[i])) * S + l;
            s_col[slot] = col[k];
            s_val[slot] = val[k];
        }
    }
}

/* SELL-P -> CSR: drop padding, keep slot order. */
void orc_sellp_to_csr(int64_t n, int64_t S, const int32_t *slice_len,
                      const int32_t *slice_set, const int32_t *s_col,
                      const double *s_val, int32_t *row_ptr, int32_t *col_out,
                      double *val_out)
{
    int64_t nz = 0;
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t s_id = i / S, l = i % S;
        for (int64_t k = 0; k < slice_len[s_id]; ++k) {
            int64_t slot = ((int64_t)slice_set[s_id] + k) * S + l;
            if (s_col[slot] < 0)
                continue;
            col_out[nz] = s_col[slot];
            val_out[nz] = s_val[slot];
            ++nz;
        }
        row_ptr[i + 1] = (int32_t)nz;
    }
}

/* Hybrid width: K_h = argmin over K in [0, max row length] of the bytes
 * n_pad * K * (s_v + 4) + overflow(K) * (s_v + 8), overflow(K) =
 * sum_i max(0, len_i - K); ties go to the smaller K.  s_v is the value size
 * in bytes. */
int64_t orc_hybrid_width(int64_t n, const int32_t *row_ptr, int64_t s_v)
{
    int64_t kmax = orc_max_row_len(n, row_ptr);
    int64_t n_pad = orc_ell_n_pad(n);
    int64_t best_k = 0;
    double best = -1.0;
    for (int64_t K = 0; K <= kmax; ++K) {
        int64_t over = 0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t L = row_ptr[i + 1] - row_ptr[i];
            if (L > K)
                over += L - K;
        }
        double bytes = (double)n_pad * (double)K * (double)(s_v + 4) +
                       (double)over * (double)(s_v + 8);
        if (best < 0.0 || bytes < best) {
            best = bytes;
            best_k = K;
        }
    }
    return best_k;
}

/* Number of entries that overflow an ELL part of width K. */
int64_t orc_hybrid_coo_nnz(int64_t n, const int32_t *row_ptr, int64_t K)
{
    int64_t over = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t L = row_ptr[i + 1] - row_ptr[i];
        if (L > K)
            over += L - K;
    }
    return over;
}

/* CSR -> hybrid: row i's first min(len_i, K) entries go to the ELL part,
 * the remaining ones, in order, to the COO part (sorted by (row, col)). */
void orc_csr_to_hybrid(int64_t n, int64_t n_pad, int64_t K, const int32_t *row_ptr,
                       const int32_t *col, const double *val, int32_t *ell_col,
                       double *ell_val, int32_t *coo_row, int32_t *coo_col,
                       double *coo_val)
{
    for (int64_t k = 0; k < K; ++k)
        for (int64_t i = 0; i < n_pad; ++i) {
            ell_col[k * n_pad + i] = -1;
            ell_val[k * n_pad + i] = 0.0;
        }
    int64_t nz = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = k - row_ptr[i];
            if (j < K) {
                ell_col[j * n_pad + i] = col[k];
                ell_val[j * n_pad + i] = val[k];
            } else {
                coo_row[nz] = (int32_t)i;
                coo_col[nz] = col[k];
                coo_val[nz] = val[k];
                ++nz;
            }
        }
}

/* hybrid -> CSR: per row, its ELL slots (padding dropped) then its COO
 * entries. */
void orc_hybrid_to_csr(int64_t n, int64_t n_pad, int64_t K, const int32_t *ell_col,
                       const double *ell_val, int64_t coo_nnz, const int32_t *coo_row,
                       const int32_t *coo_col, const double *coo_val, int32_t *row_ptr,
                       int32_t *col_out, double *val_out)
{
    int64_t nz = 0, q = 0;
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = 0; k < K; ++k) {
            int64_t slot = k * n_pad + i;
            if (ell_col[slot] < 0)
                continue;
            col_out[nz] = ell_col[slot];
            val_out[nz] = ell_val[slot];
            ++nz;
        }
        while (q < coo_nnz && coo_row[q] == i) {
            col_out[nz] = coo_col[q];
            val_out[nz] = coo_val[q];
            ++nz;
            ++q;
        }
        row_ptr[i + 1] = (int32_t)nz;
    }
}

/* ---------------------------------------------------------------- BLAS-1 */

/* Plain dot product, summed in index order. */
double orc_dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double p = a[i] * b[i];
        s = s + p;
    }
    return s;
}

/* Dot2 of Ogita-Rump-Oishi (compensated dot product). */
double orc_dot2(int64_t n, const double *a, const double *b)
{
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double p, e1, e2;
        two_prod(a[i], b[i], &p, &e1);
        two_sum(s, p, &s, &e2);
        c = c + (e1 + e2);
    }
    return s + c;
}

static double nrm2(int64_t n, const double *a) { return sqrt(orc_dot(n, a, a)); }

/* ||b - A x||_2 / ||b||_2 with the residual formed in FP64. */
double orc_true_rel_residual(int64_t n, const int32_t *row_ptr, const int32_t *col,
                             const double *val, const double *b, const double *x)
{
    double *r = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        r[i] = b[i];
    orc_spmv_csr(n, row_ptr, col, val, x, -1.0, 1.0, r);
    double nb = nrm2(n, b);
    double res = nb > 0.0 ? nrm2(n, r) / nb : nrm2(n, r);
    free(r);
    return res;
}

/* Multiple right-hand sides: Y = alpha A X + beta Y for dense blocks X
 * (n_cols x k) and Y (n_rows x k) stored row-major with leading dimensions
 * ldx, ldy: column c of the block is the product of A with column c of X,
 * each summed as orc_spmv_csr sums a row (ascending column order, separate
 * multiply and add).  beta == 0: Y is not read. */
void orc_spmm_csr(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
                  int64_t k, const double *x, int64_t ldx, double alpha, double beta, double *y,
                  int64_t ldy)
{
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t c = 0; c < k; ++c) {
            double s = 0.0;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                double t = val[e] * x[(int64_t)col[e] * ldx + c];
                s = s + t;
            }
            double out = alpha * s;
            if (beta != 0.0) {
                double u = beta * y[i * ldy + c];
                out = out + u;
            }
            y[i * ldy + c] = out;
        }
    }
}

/* ------------------------------------------------------------------- CG */

/* Conjugate gradients (Hestenes and Stiefel 1952), the Krylov solver of
 * Sec. 6.2 built on SpMV:
 *   r = b - A x0, p = r, rho = r.r
 *   repeat: q = A p; alpha = rho / (p.q); x += alpha p; r -= alpha q;
 *           rho' = r.r; beta = rho' / rho; p = r + beta p; rho = rho'.
 * Stopping: when the recursive residual satisfies sqrt(rho') <= tol ||b||,
 * the true residual ||b - A x|| / ||b|| is formed in FP64; if it is <= tol
 * the solve has converged, otherwise iteration continues; after the fourth
 * failed confirmation the solve stops with ORC_NOT_CONVERGED, as it does at
 * maxit.  p.q <= 0 (or NaN) is a breakdown (A not SPD).  ||b|| = 0 gives
 * x = 0 at once.  x holds the initial guess on entry.  *iters counts the
 * products q = A p. */
int orc_cg(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
           const double *b, double *x, double tol, int maxit, int *iters,
           double *rel_res)
{
    double nb = nrm2(n, b);
    *iters = 0;
    if (nb == 0.0) {
        for (int64_t i = 0; i < n; ++i)
            x[i] = 0.0;
        *rel_res = 0.0;
        return ORC_OK;
    }
    size_t bytes = (size_t)(n > 0 ? n : 1) * sizeof(double);
    double *r = (double *)malloc(bytes), *p = (double *)malloc(bytes),
           *q = (double *)malloc(bytes);
    for (int64_t i = 0; i < n; ++i)
        r[i] = b[i];
    orc_spmv_csr(n, row_ptr, col, val, x, -1.0, 1.0, r);
    for (int64_t i = 0; i < n; ++i)
        p[i] = r[i];
    double rho = orc_dot(n, r, r);
    int status = ORC_NOT_CONVERGED, checks = 0;
    if (sqrt(rho) <= tol * nb) {
        status = ORC_OK;
        maxit = 0;
    }
    for (int it = 0; it < maxit; ++it) {
        orc_spmv_csr(n, row_ptr, col, val, p, 1.0, 0.0, q);
        *iters = it + 1;
        double pq = orc_dot(n, p, q);
        if (!(pq > 0.0)) {
            status = ORC_BREAKDOWN;
            break;
        }
        double alpha = rho / pq;
        for (int64_t i = 0; i < n; ++i) {
            double t = alpha * p[i];
            x[i] = x[i] + t;
            double u = alpha * q[i];
            r[i] = r[i] - u;
        }
        double rho_new = orc_dot(n, r, r);
        if (!(rho_new == rho_new)) {
            status = ORC_BREAKDOWN;
            break;
        }
        if (sqrt(rho_new) <= tol * nb) {
            double t = orc_true_rel_residual(n, row_ptr, col, val, b, x);
            ++checks;
            if (t <= tol) {
                status = ORC_OK;
                break;
            }
            if (checks >= 4)
                break;
        }
        double beta = rho_new / rho;
        for (int64_t i = 0; i < n; ++i) {
            double t = beta * p[i];
            p[i] = r[i] + t;
        }
        rho = rho_new;
    }
    *rel_res = orc_true_rel_residual(n, row_ptr, col, val, b, x);
    free(r);
    free(p);
    free(q);
    return status;
}

/* CG in the single-reduction form of Chronopoulos and Gear ("s-step
 * iterative methods for symmetric linear systems", J. Comput. Appl. Math.
 * 25, 1989, with s = 1): the residual's product w = A r and the two inner
 * products gamma = r.r and delta = w.r are formed together, and the search
 * direction's product s = A p is carried by a recurrence:
 *   r = b - A x0, p = 0, s = 0
 *   repeat: w = A r; gamma = r.r; delta = w.r
 *           beta = gamma / gamma_old              (0 at the first step)
 *           alpha = gamma / (delta - beta gamma / alpha_old)
 *                                                 (gamma / delta at the first step)
 *           p = r + beta p; s = w + beta s; x += alpha p; r -= alpha s
 * In exact arithmetic the iterates equal orc_cg's.  Stopping is tested on
 * gamma of the current residual, with the same true-residual confirmation
 * as orc_cg (an unconfirmed test lets the step proceed); a non-positive or
 * NaN denominator is a breakdown.  *iters counts the updates of x. */
int orc_cg_single_reduction(int64_t n, const int32_t *row_ptr, const int32_t *col,
                            const double *val, const double *b, double *x, double tol,
                            int maxit, int *iters, double *rel_res)
{
    double nb = nrm2(n, b);
    *iters = 0;
    if (nb == 0.0) {
        for (int64_t i = 0; i < n; ++i)
            x[i] = 0.0;
        *rel_res = 0.0;
        return ORC_OK;
    }
    size_t bytes = (size_t)(n > 0 ? n : 1) * sizeof(double);
    double *r = (double *)malloc(bytes), *p = (double *)malloc(bytes),
           *s = (double *)malloc(bytes), *w = (double *)malloc(bytes);
    for (int64_t i = 0; i < n; ++i) {
        r[i] = b[i];
        p[i] = 0.0;
        s[i] = 0.0;
    }
    orc_spmv_csr(n, row_ptr, col, val, x, -1.0, 1.0, r);
    int status = ORC_NOT_CONVERGED, checks = 0, k = 0;
    double gamma_old = 0.0, alpha_old = 0.0;
    while (1) {
        orc_spmv_csr(n, row_ptr, col, val, r, 1.0, 0.0, w);
        double gamma = orc_dot(n, r, r);
        double delta = orc_dot(n, w, r);
        if (!(gamma == gamma) || !(delta == delta)) {
            status = ORC_BREAKDOWN;
            break;
        }
        if (sqrt(gamma) <= tol * nb) {
            double t = orc_true_rel_residual(n, row_ptr, col, val, b, x);
            ++checks;
            if (t <= tol) {
                status = ORC_OK;
                break;
            }
            if (checks >= 4)
                break;
        }
        if (k >= maxit)
            break;
        double beta = 0.0, denom = delta;
        if (k > 0) {
            beta = gamma / gamma_old;
            denom = delta - beta * gamma / alpha_old;
        }
        if (!(denom > 0.0)) {
            status = ORC_BREAKDOWN;
            break;
        }
        double alpha = gamma / denom;
        for (int64_t i = 0; i < n; ++i) {
            double t = beta * p[i];
            p[i] = r[i] + t;
            t = beta * s[i];
            s[i] = w[i] + t;
            t = alpha * p[i];
            x[i] = x[i] + t;
            t = alpha * s[i];
            r[i] = r[i] - t;
        }
        gamma_old = gamma;
        alpha_old = alpha;
        k += 1;
        *iters = k;
    }
    *rel_res = orc_true_rel_residual(n, row_ptr, col, val, b, x);
    free(r);
    free(p);
    free(s);
    free(w);
    return status;
}

/* CG preconditioned by the diagonal of A (Jacobi preconditioner, M = D):
 * the textbook preconditioned conjugate gradient method (e.g. Saad,
 * "Iterative Methods for Sparse Linear Systems", 2nd ed., Alg. 9.1):
 *   r = b - A x0, z = D^-1 r, p = z, rho = r.z
 *   repeat: q = A p; alpha = rho / (p.q); x += alpha p; r -= alpha q;
 *           z = D^-1 r; rho' = r.z; beta = rho' / rho; p = z + beta p.
 * Stopping on the unpreconditioned recursive residual ||r|| <= tol ||b||,
 * with the same true-residual confirmation as orc_cg.  A zero or missing
 * diagonal entry, a non-positive p.q or a NaN is a breakdown.  *iters
 * counts the products q = A p. */
int orc_pcg_jacobi(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
                   const double *b, double *x, double tol, int maxit, int *iters, double *rel_res)
{
    double nb = nrm2(n, b);
    *iters = 0;
    if (nb == 0.0) {
        for (int64_t i = 0; i < n; ++i)
            x[i] = 0.0;
        *rel_res = 0.0;
        return ORC_OK;
    }
    size_t bytes = (size_t)(n > 0 ? n : 1) * sizeof(double);
    double *r = (double *)malloc(bytes), *p = (double *)malloc(bytes),
           *q = (double *)malloc(bytes), *z = (double *)malloc(bytes),
           *d = (double *)malloc(bytes);
    int status = ORC_NOT_CONVERGED, checks = 0;
    for (int64_t i = 0; i < n; ++i) {
        d[i] = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            if (col[k] == i)
                d[i] = val[k];
        if (!(d[i] != 0.0))
            status = ORC_BREAKDOWN;
    }
    if (status == ORC_BREAKDOWN)
        maxit = 0;
    for (int64_t i = 0; i < n; ++i)
        r[i] = b[i];
    orc_spmv_csr(n, row_ptr, col, val, x, -1.0, 1.0, r);
    for (int64_t i = 0; i < n; ++i) {
        z[i] = r[i] / d[i];
        p[i] = z[i];
    }
    double rho = orc_dot(n, r, z);
    if (status != ORC_BREAKDOWN && sqrt(orc_dot(n, r, r)) <= tol * nb) {
        status = ORC_OK;
        maxit = 0;
    }
    for (int it = 0; it < maxit; ++it) {
        orc_spmv_csr(n, row_ptr, col, val, p, 1.0, 0.0, q);
        *iters = it + 1;
        double pq = orc_dot(n, p, q);
        if (!(pq > 0.0)) {
            status = ORC_BREAKDOWN;
            break;
        }
        double alpha = rho / pq;
        for (int64_t i = 0; i < n; ++i) {
            double t = alpha * p[i];
            x[i] = x[i] + t;
            double u = alpha * q[i];
            r[i] = r[i] - u;
            z[i] = r[i] / d[i];
        }
        double rr = orc_dot(n, r, r);
        double rho_new = orc_dot(n, r, z);
        if (!(rr == rr) || !(rho_new == rho_new)) {
            status = ORC_BREAKDOWN;
            break;
        }
        if (sqrt(rr) <= tol * nb) {
            double t = orc_true_rel_residual(n, row_ptr, col, val, b, x);
            ++checks;
            if (t <= tol) {
                status = ORC_OK;
                break;
            }
            if (checks >= 4)
                break;
        }
        double beta = rho_new / rho;
        for (int64_t i = 0; i < n; ++i) {
            double t = beta * p[i];
            p[i] = z[i] + t;
        }
        rho = rho_new;
    }
    *rel_res = orc_true_rel_residual(n, row_ptr, col, val, b, x);
    free(r);
    free(p);
    free(q);
    free(z);
    free(d);
    return status;
}

/* ---------------------------------------------------- block-Jacobi
 * A block-Jacobi preconditioner M = blockdiag(A_11, ..., A_kk), the
 * diagonal blocks of A on runs of consecutive rows, applied as
 * z = M^-1 r.  The paper benchmarks Krylov solvers (Sec. 6.2) without
 * defining a preconditioner; this is the textbook block-Jacobi (Saad,
 * Iterative Methods for Sparse Linear Systems, 2nd ed., Sec. 10.2, with the
 * blocks chosen as below).
 *
 * Blocks, in two steps:
 *   1. supervariables: maximal runs of consecutive rows whose stored column
 *      index lists are identical (same length, same indices in the same
 *      order), cut into pieces of at most max_bs rows (full pieces first);
 *   2. agglomeration: in row order, each piece joins the current block when
 *      the block then has at most max_bs rows, else it opens a new block.
 * block_ptr receives n_blocks + 1 boundaries (room for n + 1). */
static int same_pattern(const int32_t *row_ptr, const int32_t *col, int64_t a, int64_t b)
{
    int64_t la = row_ptr[a + 1] - row_ptr[a], lb = row_ptr[b + 1] - row_ptr[b];
    if (la != lb)
        return 0;
    for (int64_t k = 0; k < la; ++k)
        if (col[row_ptr[a] + k] != col[row_ptr[b] + k])
            return 0;
    return 1;
}

int orc_bj_blocks(int64_t n, const int32_t *row_ptr, const int32_t *col, int max_bs, int32_t *block_ptr,
                  int64_t *n_blocks)
{
    if (max_bs < 1 || max_bs > 32)
        return ORC_INVALID;
    /* step 1: the starts of the supervariable pieces, then a sentinel n */
    int64_t *piece = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t n_pieces = 0;
    for (int64_t i = 0; i < n; ++i) {
        int starts = i == 0 || !same_pattern(row_ptr, col, i - 1, i) ||
                     i - piece[n_pieces - 1] == max_bs;
        if (starts)
            piece[n_pieces++] = i;
    }
    piece[n_pieces] = n;
    /* step 2: greedy agglomeration of consecutive pieces */
    int64_t nb = 0;
    block_ptr[0] = 0;
    for (int64_t v = 0; v < n_pieces; ++v) {
        int64_t end = piece[v + 1];
        if (end - block_ptr[nb] > max_bs) { /* the piece opens a new block */
            ++nb;
            block_ptr[nb] = (int32_t)piece[v];
        }
    }
    if (n > 0) {
        ++nb;
        block_ptr[nb] = (int32_t)n;
    }
    *n_blocks = nb;
    free(piece);
    return ORC_OK;
}

/* The inverse of every diagonal block B (rows and columns o .. o+s-1 of A,
 * duplicates summed), by Gauss-Jordan elimination with partial pivoting on
 * [B | I] (Golub and Van Loan, Matrix Computations, Sec. 3.4): for each
 * column c the row of largest |B(i, c)|, i >= c, is swapped into row c,
 * row c is divided by the pivot, and c is eliminated from every other row.
 * Layout: entry (i, j) of the inverse of the block starting at row o with
 * s rows is inv[o * max_bs + j * s + i] (n * max_bs doubles in all).  A
 * zero pivot (a singular block) returns ORC_BREAKDOWN. */
int orc_bj_invert(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val, int max_bs,
                  const int32_t *block_ptr, int64_t n_blocks, double *inv)
{
    double B[32][32], E[32][32];
    (void)n;
    for (int64_t k = 0; k < n_blocks; ++k) {
        int64_t o = block_ptr[k];
        int s = (int)(block_ptr[k + 1] - o);
        for (int i = 0; i < s; ++i)
            for (int j = 0; j < s; ++j) {
                B[i][j] = 0.0;
                E[i][j] = i == j ? 1.0 : 0.0;
            }
        for (int i = 0; i < s; ++i)
            for (int64_t e = row_ptr[o + i]; e < row_ptr[o + i + 1]; ++e)
                if (col[e] >= o && col[e] < o + s)
                    B[i][col[e] - o] += val[e];
        for (int c = 0; c < s; ++c) {
            int p = c;
            for (int i = c + 1; i < s; ++i)
                if (fabs(B[i][c]) > fabs(B[p][c]))
                    p = i;
            if (B[p][c] == 0.0)
                return ORC_BREAKDOWN;
            for (int j = 0; j < s; ++j) {
                double t = B[c][j];
                B[c][j] = B[p][j];
                B[p][j] = t;
                t = E[c][j];
                E[c][j] = E[p][j];
                E[p][j] = t;
            }
            double piv = B[c][c];
            for (int j = 0; j < s; ++j) {
                B[c][j] = B[c][j] / piv;
                E[c][j] = E[c][j] / piv;
            }
            for (int i = 0; i < s; ++i) {
                if (i == c)
                    continue;
                double f = B[i][c];
                for (int j = 0; j < s; ++j) {
                    B[i][j] = B[i][j] - f * B[c][j];
                    E[i][j] = E[i][j] - f * E[c][j];
                }
            }
        }
        for (int i = 0; i < s; ++i)
            for (int j = 0; j < s; ++j)
                inv[o * max_bs + (int64_t)j * s + i] = E[i][j];
    }
    return ORC_OK;
}

/* z = M^-1 r, block by block: z(o+i) = sum_j inv(i, j) r(o+j). */
void orc_bj_apply(int max_bs, const int32_t *block_ptr, int64_t n_blocks, const double *inv, const double *r,
                  double *z)
{
    for (int64_t k = 0; k < n_blocks; ++k) {
        int64_t o = block_ptr[k];
        int s = (int)(block_ptr[k + 1] - o);
        for (int i = 0; i < s; ++i) {
            double acc = 0.0;
            for (int j = 0; j < s; ++j)
                acc = acc + inv[o * max_bs + (int64_t)j * s + i] * r[o + j];
            z[o + i] = acc;
        }
    }
}

/* Preconditioned CG (Saad, Algorithm 9.1) with the block-Jacobi M above:
 *   r = b - A x, z = M^-1 r, p = z, rho = r.z
 *   repeat: q = A p; alpha = rho / (p.q); x += alpha p; r -= alpha q;
 *           stop when ||r|| <= tol ||b|| (true-residual confirmation as in
 *           orc_cg); z = M^-1 r; rho' = r.z; p = z + (rho'/rho) p
 * A singular diagonal block is a breakdown before any step, as are a
 * non-positive p.q and a NaN.  *iters counts the products q = A p. */
int orc_pcg_block_jacobi(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val, int max_bs,
                         const double *b, double *x, double tol, int maxit, int *iters, double *rel_res)
{
    double nb = nrm2(n, b);
    *iters = 0;
    if (max_bs < 1 || max_bs > 32)
        return ORC_INVALID;
    if (nb == 0.0) {
        for (int64_t i = 0; i < n; ++i)
            x[i] = 0.0;
        *rel_res = 0.0;
        return ORC_OK;
    }
    size_t bytes = (size_t)(n > 0 ? n : 1) * sizeof(double);
    double *r = (double *)malloc(bytes), *p = (double *)malloc(bytes), *q = (double *)malloc(bytes),
           *z = (double *)malloc(bytes), *inv = (double *)malloc(bytes * (size_t)max_bs);
    int32_t *bp = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int64_t n_blocks = 0;
    int status = ORC_NOT_CONVERGED, checks = 0;
    orc_bj_blocks(n, row_ptr, col, max_bs, bp, &n_blocks);
    if (orc_bj_invert(n, row_ptr, col, val, max_bs, bp, n_blocks, inv) != ORC_OK) {
        status = ORC_BREAKDOWN;
        maxit = 0;
    }
    for (int64_t i = 0; i < n; ++i)
        r[i] = b[i];
    orc_spmv_csr(n, row_ptr, col, val, x, -1.0, 1.0, r);
    double rho = 0.0;
    if (status != ORC_BREAKDOWN) {
        orc_bj_apply(max_bs, bp, n_blocks, inv, r, z);
        for (int64_t i = 0; i < n; ++i)
            p[i] = z[i];
        rho = orc_dot(n, r, z);
        if (sqrt(orc_dot(n, r, r)) <= tol * nb) {
            status = ORC_OK;
            maxit = 0;
        }
    }
    for (int it = 0; it < maxit; ++it) {
        orc_spmv_csr(n, row_ptr, col, val, p, 1.0, 0.0, q);
        *iters = it + 1;
        double pq = orc_dot(n, p, q);
        if (!(pq > 0.0)) {
            status = ORC_BREAKDOWN;
            break;
        }
        double alpha = rho / pq;
        for (int64_t i = 0; i < n; ++i) {
            double t = alpha * p[i];
            x[i] = x[i] + t;
            double u = alpha * q[i];
            r[i] = r[i] - u;
        }
        double rr = orc_dot(n, r, r);
        if (!(rr == rr)) {
            status = ORC_BREAKDOWN;
            break;
        }
        if (sqrt(rr) <= tol * nb) {
            double t = orc_true_rel_residual(n, row_ptr, col, val, b, x);
            ++checks;
            if (t <= tol) {
                status = ORC_OK;
                break;
            }
            if (checks >= 4)
                break;
        }
        orc_bj_apply(max_bs, bp, n_blocks, inv, r, z);
        double rho_new = orc_dot(n, r, z);
        if (!(rho_new == rho_new)) {
            status = ORC_BREAKDOWN;
            break;
        }
        double beta = rho_new / rho;
        for (int64_t i = 0; i < n; ++i) {
            double t = beta * p[i];
            p[i] = z[i] + t;
        }
        rho = rho_new;
    }
    *rel_res = orc_true_rel_residual(n, row_ptr, col, val, b, x);
    free(r);
    free(p);
    free(q);
    free(z);
    free(inv);
    free(bp);
    return status;
}

/* BiCGSTAB (van der Vorst, "Bi-CGSTAB: a fast and smoothly converging
 * variant of Bi-CG for the solution of nonsymmetric linear systems", SISC
 * 13, 1992) for general square A, shadow residual r^ = r0:
 *   r = b - A x0, r^ = r, rho = alpha = omega = 1, v = p = 0
 *   repeat: rho' = r^.r; beta = (rho'/rho)(alpha/omega); p = r + beta (p - omega v)
 *           v = A p; alpha = rho' / (r^.v); s = r - alpha v
 *           if ||s|| <= tol ||b||: x += alpha p, stop (half step)
 *           t = A s; omega = (t.s)/(t.t); x += alpha p + omega s; r = s - omega t
 *           rho = rho'
 * Stopping on the recursive residual with the true-residual confirmation of
 * orc_cg; rho' = 0, r^.v = 0, t.t = 0 (or omega = 0) or a NaN is a
 * breakdown.  *iters counts full and half steps (each half step one
 * product, a full step two). */
int orc_bicgstab(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
                 const double *b, double *x, double tol, int maxit, int *iters, double *rel_res)
{
    double nb = nrm2(n, b);
    *iters = 0;
    if (nb == 0.0) {
        for (int64_t i = 0; i < n; ++i)
            x[i] = 0.0;
        *rel_res = 0.0;
        return ORC_OK;
    }
    size_t bytes = (size_t)(n > 0 ? n : 1) * sizeof(double);
    double *r = (double *)malloc(bytes), *rh = (double *)malloc(bytes), *p = (double *)malloc(bytes),
           *v = (double *)malloc(bytes), *sv = (double *)malloc(bytes), *t = (double *)malloc(bytes);
    for (int64_t i = 0; i < n; ++i)
        r[i] = b[i];
    orc_spmv_csr(n, row_ptr, col, val, x, -1.0, 1.0, r);
    for (int64_t i = 0; i < n; ++i) {
        rh[i] = r[i];
        p[i] = 0.0;
        v[i] = 0.0;
    }
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    int status = ORC_NOT_CONVERGED, checks = 0;
    if (nrm2(n, r) <= tol * nb) {
        status = ORC_OK;
        maxit = 0;
    }
    for (int it = 0; it < maxit; ++it) {
        double rho_new = orc_dot(n, rh, r);
        if (!(rho_new != 0.0) || !(rho_new == rho_new)) {
            status = ORC_BREAKDOWN;
            break;
        }
        double beta = (rho_new / rho) * (alpha / omega);
        for (int64_t i = 0; i < n; ++i) {
            double u = omega * v[i];
            double w = p[i] - u;
            double z = beta * w;
            p[i] = r[i] + z;
        }
        orc_spmv_csr(n, row_ptr, col, val, p, 1.0, 0.0, v);
        double rv = orc_dot(n, rh, v);
        if (!(rv != 0.0) || !(rv == rv)) {
            status = ORC_BREAKDOWN;
            break;
        }
        alpha = rho_new / rv;
        for (int64_t i = 0; i < n; ++i) {
            double u = alpha * v[i];
            sv[i] = r[i] - u;
        }
        *iters = it + 1;
        if (nrm2(n, sv) <= tol * nb) { /* half step */
            for (int64_t i = 0; i < n; ++i) {
                double u = alpha * p[i];
                x[i] = x[i] + u;
            }
            double tr = orc_true_rel_residual(n, row_ptr, col, val, b, x);
            ++checks;
            if (tr <= tol) {
                status = ORC_OK;
                break;
            }
            if (checks >= 4)
                break;
            /* unconfirmed: restart from the true residual of this iterate */
            for (int64_t i = 0; i < n; ++i)
                r[i] = b[i];
            orc_spmv_csr(n, row_ptr, col, val, x, -1.0, 1.0, r);
            for (int64_t i = 0; i < n; ++i) {
                rh[i] = r[i];
                p[i] = 0.0;
                v[i] = 0.0;
            }
            rho = alpha = omega = 1.0;
            continue;
        }
        orc_spmv_csr(n, row_ptr, col, val, sv, 1.0, 0.0, t);
        double tt = orc_dot(n, t, t);
        double ts = orc_dot(n, t, sv);
        if (!(tt > 0.0) || !(ts == ts)) {
            status = ORC_BREAKDOWN;
            break;
        }
        omega = ts / tt;
        if (!(omega != 0.0)) {
            status = ORC_BREAKDOWN;
            break;
        }
        for (int64_t i = 0; i < n; ++i) {
            double u = alpha * p[i];
            double w = omega * sv[i];
            x[i] = x[i] + u;
            x[i] = x[i] + w;
            double z = omega * t[i];
            r[i] = sv[i] - z;
        }
        rho = rho_new;
        double nr = nrm2(n, r);
        if (!(nr == nr)) {
            status = ORC_BREAKDOWN;
            break;
        }
        if (nr <= tol * nb) {
            double tr = orc_true_rel_residual(n, row_ptr, col, val, b, x);
            ++checks;
            if (tr <= tol) {
                status = ORC_OK;
                break;
            }
            if (checks >= 4)
                break;
        }
    }
    *rel_res = orc_true_rel_residual(n, row_ptr, col, val, b, x);
    free(r);
    free(rh);
    free(p);
    free(v);
    free(sv);
    free(t);
    return status;
}

/* Restarted GMRES(m) (Saad and Schultz, SISC 7, 1986) for general square
 * A: each cycle builds the Arnoldi basis v_1 = r/||r||, v_{j+1} from A v_j
 * orthogonalised against v_1..v_j by modified Gram-Schmidt, reduces the
 * Hessenberg matrix to triangular form by Givens rotations (whose last
 * right-hand side entry is the residual norm of the least-squares
 * minimiser), stops the cycle at j = m or when that norm is <= tol ||b||,
 * solves the triangular system and updates x; then r = b - A x (the true
 * residual) starts the next cycle.  Converged when the true residual
 * confirms; *iters counts Arnoldi steps (products with A after the first
 * residual of each cycle).  A zero subdiagonal before convergence (lucky
 * breakdown) ends the cycle with the exact solution of the subspace. */
int orc_gmres(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
              const double *b, double *x, double tol, int m, int maxit, int *iters,
              double *rel_res)
{
    double nb = nrm2(n, b);
    *iters = 0;
    if (nb == 0.0) {
        for (int64_t i = 0; i < n; ++i)
            x[i] = 0.0;
        *rel_res = 0.0;
        return ORC_OK;
    }
    if (m < 1)
        m = 1;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *V = (double *)malloc(nn * (size_t)(m + 1) * sizeof(double));
    double *r = (double *)malloc(nn * sizeof(double)), *w = (double *)malloc(nn * sizeof(double));
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double *cs = (double *)malloc((size_t)m * sizeof(double)), *sn = (double *)malloc((size_t)m * sizeof(double));
    double *g = (double *)malloc((size_t)(m + 1) * sizeof(double)), *yv = (double *)malloc((size_t)m * sizeof(double));
    int status = ORC_NOT_CONVERGED, total = 0;
    while (1) {
        for (int64_t i = 0; i < n; ++i)
            r[i] = b[i];
        orc_spmv_csr(n, row_ptr, col, val, x, -1.0, 1.0, r);
        double beta = nrm2(n, r);
        if (!(beta == beta)) {
            status = ORC_BREAKDOWN;
            break;
        }
        if (beta <= tol * nb) {
            status = ORC_OK;
            break;
        }
        if (total >= maxit)
            break;
        for (int64_t i = 0; i < n; ++i)
            V[i] = r[i] / beta;
        for (int k = 0; k <= m; ++k)
            g[k] = 0.0;
        g[0] = beta;
        int j = 0;
        for (; j < m && total < maxit; ++j) {
            orc_spmv_csr(n, row_ptr, col, val, V + (size_t)j * nn, 1.0, 0.0, w);
            total += 1;
            for (int i = 0; i <= j; ++i) { /* modified Gram-Schmidt */
                double h = orc_dot(n, w, V + (size_t)i * nn);
                H[(size_t)i * m + j] = h;
                for (int64_t q = 0; q < n; ++q) {
                    double t = h * V[(size_t)i * nn + q];
                    w[q] = w[q] - t;
                }
            }
            double hn = nrm2(n, w);
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (int64_t q = 0; q < n; ++q)
                    V[(size_t)(j + 1) * nn + q] = w[q] / hn;
            for (int i = 0; i < j; ++i) { /* earlier rotations on the new column */
                double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
            double d = sqrt(a * a + c * c);
            if (!(d > 0.0)) {
                status = ORC_BREAKDOWN;
                break;
            }
            cs[j] = a / d;
            sn[j] = c / d;
            H[(size_t)j * m + j] = d;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (fabs(g[j + 1]) <= tol * nb || !(hn > 0.0)) {
                j += 1;
                break;
            }
        }
        if (status == ORC_BREAKDOWN)
            break;
        for (int i = j - 1; i >= 0; --i) { /* back substitution */
            double s = g[i];
            for (int k = i + 1; k < j; ++k) {
                double t = H[(size_t)i * m + k] * yv[k];
                s = s - t;
            }
            yv[i] = s / H[(size_t)i * m + i];
        }
        for (int i = 0; i < j; ++i)
            for (int64_t q = 0; q < n; ++q) {
                double t = yv[i] * V[(size_t)i * nn + q];
                x[q] = x[q] + t;
            }
    }
    *iters = total;
    *rel_res = orc_true_rel_residual(n, row_ptr, col, val, b, x);
    free(V);
    free(r);
    free(w);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(yv);
    return status;
}

/* Batched CG: systems s = 0..count-1 with rows [row_off[s], row_off[s+1])
 * of one concatenated CSR whose row_ptr is global and whose column indices
 * are local to the system.  Each system is solved by orc_cg. */
int orc_cg_batched(int64_t count, const int64_t *row_off, const int32_t *row_ptr,
                   const int32_t *col, const double *val, const double *b, double *x,
                   double tol, int maxit, int *iters, double *rel_res, int *status)
{
    int worst = ORC_OK;
    for (int64_t s = 0; s < count; ++s) {
        int64_t r0 = row_off[s], n = row_off[s + 1] - row_off[s];
        int32_t *rp = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
        for (int64_t i = 0; i <= n; ++i)
            rp[i] = row_ptr[r0 + i] - row_ptr[r0];
        status[s] = orc_cg(n, rp, col + row_ptr[r0], val + row_ptr[r0], b + r0, x + r0,
                           tol, maxit, &iters[s], &rel_res[s]);
        if (status[s] != ORC_OK)
            worst = status[s];
        free(rp);
    }
    return worst;
}

/* ------------------------------------------------- mixed precision + IR */

/* Round a double to the nearest bfloat16 (8 significant bits), ties to
 * even, returned as a double; up != 0 rounds toward +infinity instead.
 * Written from the definition: scale the significand to 8 bits with frexp,
 * round to an integer, scale back.  Values are assumed inside the normal
 * bfloat16 range. */
double orc_round_bf16(double v, int up)
{
    if (v == 0.0 || !isfinite(v))
        return v;
    int e;
    double m = frexp(v, &e); /* v = m * 2^e, 0.5 <= |m| < 1 */
    double sig = ldexp(m, 8);
    double r = up ? ceil(sig) : nearbyint(sig); /* default mode: ties-to-even */
    return ldexp(r, e - 8);
}

/* The same for binary32 (24 significant bits). */
double orc_round_fp32(double v, int up)
{
    if (v == 0.0 || !isfinite(v))
        return v;
    int e;
    double m = frexp(v, &e);
    double sig = ldexp(m, 24);
    double r = up ? ceil(sig) : nearbyint(sig);
    return ldexp(r, e - 24);
}

/* Low-precision copy of an SPD matrix (prec 1 = FP32, 2 = BF16): every
 * off-diagonal entry is rounded to nearest-even; the diagonal becomes
 * a_ii + sum_j (|rn(a_ij)| - |a_ij|), formed in FP64 (for a matrix with
 * non-positive off-diagonals this keeps every row sum of the copy equal to
 * the original's), then rounded to nearest-even.  Rounding the diagonal to
 * nearest keeps the perturbation zero-mean: an upward rounding would add a
 * one-sided shift of up to one BF16 ulp (~0.4 % of a_ii) to every row,
 * which exceeds the smallest eigenvalue of ill-conditioned diffusion
 * operators and stalls the refinement.  SPD-ness of the copy is therefore
 * not guaranteed by construction; the inner CG detects a breakdown. */
void orc_round_matrix(int64_t n, const int32_t *row_ptr, const int32_t *col,
                      const double *val, int prec, double *val_lo)
{
    for (int64_t i = 0; i < n; ++i) {
        double shift = 0.0;
        int64_t kd = -1;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (col[k] == i) {
                kd = k;
                continue;
            }
            double r = prec == 2 ? orc_round_bf16(val[k], 0) : orc_round_fp32(val[k], 0);
            val_lo[k] = r;
            double d = fabs(r) - fabs(val[k]);
            shift = shift + d;
        }
        if (kd >= 0) {
            double d = val[kd] + shift;
            val_lo[kd] = prec == 2 ? orc_round_bf16(d, 0) : orc_round_fp32(d, 0);
        }
    }
}

/* Mixed-precision CG with FP64 iterative refinement.
 * Outer loop (FP64): r = b - A x with the FP64 matrix; stop when
 * ||r|| / ||b|| <= tol; otherwise solve A_lo d = r / ||r|| approximately by
 * an inner CG in FP32 arithmetic (FP32 vectors, FP32 products and row sums on
 * the rounded matrix val_lo, dot products accumulated in FP64 and rounded
 * to FP32) to relative recursive residual inner_tol or inner_maxit steps;
 * then x += ||r|| d in FP64.  x holds the initial guess.  Counts outer
 * corrections in *outer and inner CG steps in *inner. */
int orc_cg_mixed_precond(int64_t n, const int32_t *row_ptr, const int32_t *col,
                         const double *val, const double *val_lo, const double *b, double *x,
                         double tol, int maxit_outer, double inner_tol, int inner_maxit, int precond,
                         int *outer, int *inner, double *rel_res)
{
    double nb = nrm2(n, b);
    *outer = 0;
    *inner = 0;
    if (nb == 0.0) {
        for (int64_t i = 0; i < n; ++i)
            x[i] = 0.0;
        *rel_res = 0.0;
        return ORC_OK;
    }
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *r = (double *)malloc(nn * sizeof(double));
    float *rl = (float *)malloc(nn * sizeof(float)), *d = (float *)malloc(nn * sizeof(float)),
          *p = (float *)malloc(nn * sizeof(float)), *q = (float *)malloc(nn * sizeof(float)),
          *vl = (float *)malloc((size_t)(row_ptr[n] > 0 ? row_ptr[n] : 1) * sizeof(float)),
          *z = (float *)malloc(nn * sizeof(float)), *dl = (float *)malloc(nn * sizeof(float));
    for (int64_t k = 0; k < row_ptr[n]; ++k)
        vl[k] = (float)val_lo[k]; /* exact: val_lo holds FP32/BF16 values */
    int status = ORC_NOT_CONVERGED;
    for (int64_t i = 0; i < n; ++i) { /* diagonal of A_lo (Jacobi) */
        dl[i] = 0.0f;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            if (col[k] == i)
                dl[i] = vl[k];
        if (precond && !(dl[i] != 0.0f))
            status = ORC_BREAKDOWN;
    }
    if (status == ORC_BREAKDOWN)
        maxit_outer = 0;
    for (int o = 0; o <= maxit_outer; ++o) {
        for (int64_t i = 0; i < n; ++i)
            r[i] = b[i];
        orc_spmv_csr(n, row_ptr, col, val, x, -1.0, 1.0, r);
        double nr = nrm2(n, r);
        if (nr <= tol * nb) {
            status = ORC_OK;
            break;
        }
        if (o == maxit_outer)
            break;
        *outer = o + 1;
        /* inner CG on A_lo d = r / ||r||, d0 = 0, preconditioned by
         * M = diag(A_lo) when precond (z = M^-1 r; else z = r) */
        for (int64_t i = 0; i < n; ++i) {
            rl[i] = (float)(r[i] / nr);
            d[i] = 0.0f;
            z[i] = precond ? rl[i] / dl[i] : rl[i];
            p[i] = z[i];
        }
        double rho_d = 0.0;
        for (int64_t i = 0; i < n; ++i)
            rho_d = rho_d + (double)rl[i] * (double)z[i];
        float rho = (float)rho_d;
        float rho0 = rho;
        for (int it = 0; it < inner_maxit; ++it) {
            for (int64_t i = 0; i < n; ++i) {
                float s = 0.0f;
                for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                    float t = vl[k] * p[col[k]];
                    s = s + t;
                }
                q[i] = s;
            }
            *inner += 1;
            double pq_d = 0.0;
            for (int64_t i = 0; i < n; ++i)
                pq_d = pq_d + (double)p[i] * (double)q[i];
            float pq = (float)pq_d;
            if (!(pq > 0.0f))
                break;
            float alpha = rho / pq;
            for (int64_t i = 0; i < n; ++i) {
                float t = alpha * p[i];
                d[i] = d[i] + t;
                float u = alpha * q[i];
                rl[i] = rl[i] - u;
                z[i] = precond ? rl[i] / dl[i] : rl[i];
            }
            double rn_d = 0.0;
            for (int64_t i = 0; i < n; ++i)
                rn_d = rn_d + (double)rl[i] * (double)z[i];
            float rho_new = (float)rn_d;
            if (sqrtf(rho_new) <= (float)inner_tol * sqrtf(rho0))
                break;
            float beta = rho_new / rho;
            for (int64_t i = 0; i < n; ++i) {
                float t = beta * p[i];
                p[i] = z[i] + t;
            }
            rho = rho_new;
        }
        for (int64_t i = 0; i < n; ++i) {
            double t = nr * (double)d[i];
            x[i] = x[i] + t;
        }
    }
    *rel_res = orc_true_rel_residual(n, row_ptr, col, val, b, x);
    free(r);
    free(rl);
    free(d);
    free(p);
    free(q);
    free(vl);
    free(z);
    free(dl);
    return status;
}

/* The unpreconditioned inner solve (z = r). */
int orc_cg_mixed(int64_t n, const int32_t *row_ptr, const int32_t *col,
                 const double *val, const double *val_lo, const double *b, double *x,
                 double tol, int maxit_outer, double inner_tol, int inner_maxit,
                 int *outer, int *inner, double *rel_res)
{
    return orc_cg_mixed_precond(n, row_ptr, col, val, val_lo, b, x, tol, maxit_outer, inner_tol,
                                inner_maxit, 0, outer, inner, rel_res);
}

/* ------------------------------------------------------- dense Cholesky */

/* Solve A x = b for a dense SPD A (row-major n x n) by Cholesky A = L L^T,
 * forward and back substitution.  Returns ORC_BREAKDOWN if a pivot is not
 * positive.  A is not modified. */
int orc_cholesky_solve(int64_t n, const double *A, const double *b, double *x)
{
    double *L = (double *)calloc((size_t)(n * n > 0 ? n * n : 1), sizeof(double));
    for (int64_t j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int64_t k = 0; k < j; ++k) {
            double t = L[j * n + k] * L[j * n + k];
            s = s - t;
        }
        if (!(s > 0.0)) {
            free(L);
            return ORC_BREAKDOWN;
        }
        L[j * n + j] = sqrt(s);
        for (int64_t i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int64_t k = 0; k < j; ++k) {
                double u = L[i * n + k] * L[j * n + k];
                t = t - u;
            }
            L[i * n + j] = t / L[j * n + j];
        }
    }
    for (int64_t i = 0; i < n; ++i) { /* L y = b */
        double t = b[i];
        for (int64_t k = 0; k < i; ++k) {
            double u = L[i * n + k] * x[k];
            t = t - u;
        }
        x[i] = t / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) { /* L^T x = y */
        double t = x[i];
        for (int64_t k = i + 1; k < n; ++k) {
            double u = L[k * n + i] * x[k];
            t = t - u;
        }
        x[i] = t / L[i * n + i];
    }
    free(L);
    return ORC_OK;
}

/* ------------------------------------------------------------- features */

/* The 12 matrix statistics of the format selector, in order:
 *  0 log10(n)            1 log10(max(nnz, 1))     2 mean row length
 *  3 std of row lengths  4 max row length         5 min row length
 *  6 max / mean (0 if mean is 0)                  7 fraction of empty rows
 *  8 max |i - j| / n     9 mean |i - j| / n over stored entries (0 if none)
 * 10 fraction of rows that store their diagonal
 * 11 SELL-P slots / nnz with slices of 32 rows, stride factor 1 (0 if nnz 0)
 * n = number of rows (> 0).  Standard deviation is the population one. */
void orc_features(int64_t n, const int32_t *row_ptr, const int32_t *col, double *f)
{
    int64_t nnz = row_ptr[n];
    double mean = (double)nnz / (double)n;
    double var = 0.0, maxd = 0.0, sumd = 0.0;
    int64_t lmax = 0, lmin = -1, empty = 0, diag = 0, slots = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t L = row_ptr[i + 1] - row_ptr[i];
        double dev = (double)L - mean;
        var = var + dev * dev;
        if (L > lmax)
            lmax = L;
        if (lmin < 0 || L < lmin)
            lmin = L;
        if (L == 0)
            ++empty;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            double dd = fabs((double)col[k] - (double)i);
            if (dd > maxd)
                maxd = dd;
            sumd = sumd + dd;
            if (col[k] == i)
                ++diag;
        }
    }
    for (int64_t s = 0; s * 32 < n; ++s) {
        int64_t w = 0;
        for (int64_t i = s * 32; i < s * 32 + 32 && i < n; ++i)
            if (row_ptr[i + 1] - row_ptr[i] > w)
                w = row_ptr[i + 1] - row_ptr[i];
        slots += 32 * w;
    }
    f[0] = log10((double)n);
    f[1] = log10((double)(nnz > 0 ? nnz : 1));
    f[2] = mean;
    f[3] = sqrt(var / (double)n);
    f[4] = (double)lmax;
    f[5] = (double)lmin;
    f[6] = mean > 0.0 ? (double)lmax / mean : 0.0;
    f[7] = (double)empty / (double)n;
    f[8] = maxd / (double)n;
    f[9] = nnz > 0 ? sumd / (double)nnz / (double)n : 0.0;
    f[10] = (double)diag / (double)n;
    f[11] = nnz > 0 ? (double)slots / (double)nnz : 0.0;
}
