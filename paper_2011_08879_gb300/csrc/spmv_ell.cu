// ELL, SELL-P and hybrid ELL+COO SpMV (the paper's Sec. 6.1 "distinct
// storage formats"; ELL/hybrid after Bell and Garland 2009, SELL-P after
// Anzt, Tomov and Dongarra 2014).
//
// Padded formats are column-major, so consecutive threads read consecutive
// slots: every thread owns two consecutive rows and moves their values and
// column indices with one 128-bit (double2) and one 64-bit (int2) load per
// slot.  Padding slots (col == -1) are skipped, so 0 * Inf never turns into
// NaN; each stored entry costs exactly one FP64 FMA.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "segmented.cuh"
#include "ell.cuh"

namespace gko {

int launch_seg(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row_ptr, const int32_t* rows, const int32_t* col,
               const double* val, const int32_t* thr_row, const SegArrays& sa, const double* x, double* y,
               double alpha, double beta, uint32_t* err, bool coo, cudaStream_t st, bool accumulate, int coo_p);

// Two rows per thread; slot k of rows (2p, 2p+1) at k*ld + 2p.
template <bool kAlpha, bool kBeta>
__global__ void __launch_bounds__(256)
    ell_kernel(int64_t n_rows, int64_t n_pad, int64_t K, const int32_t* __restrict__ col,
               const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y, double alpha,
               double beta)
{
    const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int64_t r = 2 * p;
    if (r >= n_rows) return;
    double a0, a1;
    ell_pair_sum(r, n_pad, K, col, val, x, a0, a1);
    store_pair<kAlpha, kBeta>(y, r, n_rows, a0, a1, alpha, beta);
}

// SELL-P: two rows per thread inside a slice of S rows (S even).
template <bool kAlpha, bool kBeta>
__global__ void __launch_bounds__(256)
    sellp_kernel(int64_t n_rows, int64_t S, const int32_t* __restrict__ slice_len,
                 const int32_t* __restrict__ slice_set, const int32_t* __restrict__ col,
                 const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y, double alpha,
                 double beta)
{
    const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int64_t r = 2 * p;
    if (r >= n_rows) return;
    const int64_t sl = r / S, l = r % S;
    const int64_t w = slice_len[sl];
    const int64_t base = static_cast<int64_t>(slice_set[sl]) * S + l;
    const int2* c2 = reinterpret_cast<const int2*>(col + base);
    const double2* v2 = reinterpret_cast<const double2*>(val + base);
    const int64_t step = S / 2;
    double a0 = 0.0, a1 = 0.0;
    int64_t k = 0;
    for (; k + 4 <= w; k += 4) {
        int2 c[4];
        double2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = __ldcs(c2 + (k + u) * step);
            v[u] = __ldcs(v2 + (k + u) * step);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u].x >= 0) a0 = fma(v[u].x, ldg(x + c[u].x), a0);
            if (c[u].y >= 0) a1 = fma(v[u].y, ldg(x + c[u].y), a1);
        }
    }
    for (; k < w; ++k) {
        const int2 c = __ldcs(c2 + k * step);
        const double2 v = __ldcs(v2 + k * step);
        if (c.x >= 0) a0 = fma(v.x, ldg(x + c.x), a0);
        if (c.y >= 0) a1 = fma(v.y, ldg(x + c.y), a1);
    }
    store_pair<kAlpha, kBeta>(y, r, n_rows, a0, a1, alpha, beta);
}

// SELL-P with S == 1 (one row per slice): one row per thread.
template <bool kAlpha, bool kBeta>
__global__ void __launch_bounds__(256)
    sellp1_kernel(int64_t n_rows, const int32_t* __restrict__ slice_len, const int32_t* __restrict__ slice_set,
                  const int32_t* __restrict__ col, const double* __restrict__ val, const double* __restrict__ x,
                  double* __restrict__ y, double alpha, double beta)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= n_rows) return;
    const int64_t w = slice_len[r], base = slice_set[r];
    double a = 0.0;
    for (int64_t k = 0; k < w; ++k) {
        const int32_t c = col[base + k];
        if (c >= 0) a = fma(val[base + k], ldg(x + c), a);
    }
    seg_store<kAlpha, kBeta>(y, r, a, alpha, beta);
}

#define GKO_AB_DISPATCH(LAUNCH)            \
    do {                                   \
        const bool _a = alpha != 1.0;      \
        const bool _b = beta != 0.0;       \
        if (_a && _b)                      \
            LAUNCH(true, true);            \
        else if (_a)                       \
            LAUNCH(true, false);           \
        else if (_b)                       \
            LAUNCH(false, true);           \
        else                               \
            LAUNCH(false, false);          \
    } while (0)

int spmv_ell(const gko_matrix* A, const EllPart& e, const double* x, double* y, double alpha, double beta,
             cudaStream_t st)
{
    const int64_t n = A->n_rows;
    if (n == 0) return GKO_OK;
    if (e.K == 0) return scale_vector(n, y, beta, st);
    const int grid = ceil_div((n + 1) / 2, 256);
#define GKO_L(KA, KB) ell_kernel<KA, KB><<<grid, 256, 0, st>>>(n, e.n_pad, e.K, e.col, e.val, x, y, alpha, beta)
    GKO_AB_DISPATCH(GKO_L);
#undef GKO_L
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

int spmv_sellp(const gko_matrix* A, const double* x, double* y, double alpha, double beta, cudaStream_t st)
{
    const SellpPart& s = A->sellp;
    const int64_t n = A->n_rows;
    if (n == 0) return GKO_OK;
    if (s.S == 1) {
        const int grid = ceil_div(n, 256);
#define GKO_L(KA, KB) \
    sellp1_kernel<KA, KB><<<grid, 256, 0, st>>>(n, s.slice_len, s.slice_set, s.col, s.val, x, y, alpha, beta)
        GKO_AB_DISPATCH(GKO_L);
#undef GKO_L
    } else {
        const int grid = ceil_div((n + 1) / 2, 256);
#define GKO_L(KA, KB) \
    sellp_kernel<KA, KB><<<grid, 256, 0, st>>>(n, s.S, s.slice_len, s.slice_set, s.col, s.val, x, y, alpha, beta)
        GKO_AB_DISPATCH(GKO_L);
#undef GKO_L
    }
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

// hybrid: y = alpha * A_ell x + beta * y, then y += alpha * A_coo x
int spmv_hybrid(const gko_matrix* A, const double* x, double* y, double alpha, double beta, cudaStream_t st)
{
    const HybridPart& h = A->hyb;
    GKO_TRY(spmv_ell(A, h.ell, x, y, alpha, beta, st));
    if (h.coo.nnz == 0) return GKO_OK;
    return launch_seg(A->n_rows, A->n_cols, h.coo.nnz, nullptr, h.coo.row, h.coo.col, h.coo.val, nullptr, h.coo.seg, x, y,
                      alpha, 1.0, A->d_err, true, st, true, h.coo.P);
}

}  // namespace gko
