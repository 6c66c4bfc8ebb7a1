// Multi-right-hand-side CSR product Y = alpha A X + beta Y for dense blocks
// X (n_cols x k) and Y (n_rows x k) stored row-major: the Krylov solvers of
// the paper's Sec. 6.2 applied to several right-hand sides at once share
// one pass over the matrix.  Gathering row j of X brings k contiguous
// doubles (whole 32-byte sectors from k = 4 on) and each stored entry's
// value and column are read once for all k columns.
//
// A subwarp of KL lanes (the power of two >= min(k, 32)) owns a row; lane l
// takes columns l, l + KL, ...: for each stored entry the subwarp reads the
// value and column once (same address: one broadcast transaction) and the KL
// consecutive entries of row col of X.  Entries go four at a time (loads,
// then gathers, then FMAs into two chains).  One FP64 FMA per (entry,
// column): on GB300 (FP64 FMA ~1/64 of the FP32 rate) the product is bound
// by the FP64 pipe from k of about 2 on, not by HBM.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "segmented.cuh"

namespace gko {

template <int KL, bool kAlpha, bool kBeta>
__global__ void __launch_bounds__(256)
    spmm_csr_kernel(int64_t n, int64_t k, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                    const double* __restrict__ val, const double* __restrict__ x, int64_t ldx, double* __restrict__ y,
                    int64_t ldy, double alpha, double beta)
{
    constexpr int kRowsPerWarp = kWarp / KL;
    const int lane = threadIdx.x % KL;
    const int sub = (threadIdx.x % kWarp) / KL;
    const int64_t warp = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) / kWarp;
    const int64_t n_warps = static_cast<int64_t>(gridDim.x) * blockDim.x / kWarp;
    for (int64_t base = warp * kRowsPerWarp; base < n; base += n_warps * kRowsPerWarp) {
        const int64_t r = base + sub;
        if (r >= n) continue;
        const int32_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
        for (int64_t c = lane; c - lane < k; c += KL) {
            const bool on = c < k;
            double a0 = 0.0, a1 = 0.0;
            int32_t e = e0;
            for (; e + 4 <= e1; e += 4) {
                int32_t j[4];
                double v[4], xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    j[u] = col[e + u];
                    v[u] = val[e + u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) xv[u] = on ? ldg(x + static_cast<int64_t>(j[u]) * ldx + c) : 0.0;
                a0 = fma(v[0], xv[0], a0);
                a1 = fma(v[1], xv[1], a1);
                a0 = fma(v[2], xv[2], a0);
                a1 = fma(v[3], xv[3], a1);
            }
            for (; e < e1; ++e) a0 = fma(val[e], on ? ldg(x + static_cast<int64_t>(col[e]) * ldx + c) : 0.0, a0);
            if (on) {
                double out = a0 + a1;
                if (kAlpha) out *= alpha;
                if (kBeta) out = fma(beta, y[r * ldy + c], out);
                y[r * ldy + c] = out;
            }
        }
    }
}

template <int KL>
static void launch_spmm_kl(const gko_matrix* A, int64_t k, const double* x, int64_t ldx, double* y, int64_t ldy,
                           double alpha, double beta, cudaStream_t st)
{
    const CsrPart& c = A->csr;
    const int64_t rows_per_block = 256 / KL;
    const int grid = static_cast<int>(std::min<int64_t>((A->n_rows + rows_per_block - 1) / rows_per_block,
                                                        152LL * 16));
    const bool a = alpha != 1.0, b = beta != 0.0;
#define GKO_MM(KA, KB)                                                                                   \
    spmm_csr_kernel<KL, KA, KB><<<grid, 256, 0, st>>>(A->n_rows, k, c.row_ptr, c.col, c.val, x, ldx, y, ldy, \
                                                      alpha, beta)
    if (a && b)
        GKO_MM(true, true);
    else if (a)
        GKO_MM(true, false);
    else if (b)
        GKO_MM(false, true);
    else
        GKO_MM(false, false);
#undef GKO_MM
}

// y[i*ldy + c] = beta * y[i*ldy + c] (beta = 0: zero) for an empty matrix
__global__ void spmm_scale_kernel(int64_t n, int64_t k, double* __restrict__ y, int64_t ldy, double beta)
{
    const int64_t total = n * k;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = t / k, c = t % k;
        y[i * ldy + c] = beta == 0.0 ? 0.0 : beta * y[i * ldy + c];
    }
}

int spmm_csr(const gko_matrix* A, int64_t k, const double* x, int64_t ldx, double* y, int64_t ldy, double alpha,
             double beta, cudaStream_t st)
{
    if (A->n_rows == 0 || k == 0) return GKO_OK;
    if (A->nnz == 0) {
        spmm_scale_kernel<<<std::min(ceil_div(A->n_rows * k, 256), 152 * 8), 256, 0, st>>>(A->n_rows, k, y, ldy,
                                                                                          beta);
    } else if (k == 1) {
        launch_spmm_kl<1>(A, k, x, ldx, y, ldy, alpha, beta, st);
    } else if (k == 2) {
        launch_spmm_kl<2>(A, k, x, ldx, y, ldy, alpha, beta, st);
    } else if (k <= 4) {
        launch_spmm_kl<4>(A, k, x, ldx, y, ldy, alpha, beta, st);
    } else if (k <= 8) {
        launch_spmm_kl<8>(A, k, x, ldx, y, ldy, alpha, beta, st);
    } else if (k <= 16) {
        launch_spmm_kl<16>(A, k, x, ldx, y, ldy, alpha, beta, st);
    } else {
        launch_spmm_kl<32>(A, k, x, ldx, y, ldy, alpha, beta, st);
    }
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

}  // namespace gko
