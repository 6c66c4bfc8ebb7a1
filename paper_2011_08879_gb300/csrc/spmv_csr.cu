// CSR SpMV (paper Sec. 6.1: y = A x in CSR, bounded by 12 bytes/entry):
//  * classical subwarp-per-row kernel (subwarp of 1..32 lanes, chosen at
//    run time; the paper's cooperative-group subwarps and Listing 2's
//    butterfly reduction);
//  * load-balanced equal-nnz kernel (segmented.cuh), the default;
//  * banded kernel: the x window of a row block staged in shared memory.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "segmented.cuh"

namespace gko {

// ------------------------------------------------------------- analysis

// thr_row[g] = the row that holds entry g*P, i.e. the first r with
// row_ptr[r+1] > g*P (rows that end at or before g*P are skipped).
__global__ void thr_row_kernel(int64_t n_rows, int64_t n_thr, int64_t P, const int32_t* __restrict__ row_ptr,
                               int32_t* __restrict__ thr_row)
{
    const int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (g >= n_thr) return;
    const int64_t v = g * P;
    int64_t lo = 0, hi = n_rows;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (row_ptr[mid + 1] <= v)
            lo = mid + 1;
        else
            hi = mid;
    }
    thr_row[g] = static_cast<int32_t>(lo);
}

// max row length and max |i - j| (from each row's first and last column)
__global__ void row_stats_kernel(int64_t n_rows, const int32_t* __restrict__ row_ptr,
                                 const int32_t* __restrict__ col, int32_t* __restrict__ out)
{
    int32_t mx = 0, band = 0;
    for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n_rows;
         r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t a = row_ptr[r], b = row_ptr[r + 1];
        mx = max(mx, b - a);
        if (b > a) {
            band = max(band, static_cast<int32_t>(abs(static_cast<int64_t>(col[a]) - r)));
            band = max(band, static_cast<int32_t>(abs(static_cast<int64_t>(col[b - 1]) - r)));
        }
    }
    for (int o = 16; o; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        band = max(band, __shfl_xor_sync(0xffffffffu, band, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, mx);
        atomicMax(out + 1, band);
    }
}

int seg_alloc(SegArrays* s, int64_t nnz, int P)
{
    seg_free(s);
    const int64_t tile = static_cast<int64_t>(kSegThreads) * P;
    s->n_tiles = (nnz + tile - 1) / tile;
    const int64_t t = std::max<int64_t>(s->n_tiles, 1);
    GKO_TRY(dev_alloc(&s->tail_val, t));
    GKO_TRY(dev_alloc(&s->tail_row, t));
    GKO_TRY(dev_alloc(&s->tail_pass, t));
    GKO_TRY(dev_alloc(&s->head_val, t));
    GKO_TRY(dev_alloc(&s->head_row, t));
    return GKO_OK;
}

void seg_free(SegArrays* s)
{
    dev_free(s->tail_val);
    dev_free(s->tail_row);
    dev_free(s->tail_pass);
    dev_free(s->head_val);
    dev_free(s->head_row);
    s->n_tiles = 0;
}

int compute_thr_row(int64_t n_rows, int64_t nnz, const int32_t* row_ptr, int32_t* thr_row, cudaStream_t st)
{
    const int64_t n_thr = (nnz + kSegP - 1) / kSegP;
    if (n_thr > 0) thr_row_kernel<<<ceil_div(n_thr, 256), 256, 0, st>>>(n_rows, n_thr, kSegP, row_ptr, thr_row);
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

int csr_analyse(gko_matrix* A, cudaStream_t st)
{
    CsrPart& c = A->csr;
    dev_free(c.thr_row);
    const int64_t n_thr = (A->nnz + kSegP - 1) / kSegP;
    GKO_TRY(dev_alloc(&c.thr_row, std::max<int64_t>(n_thr, 1)));
    if (n_thr > 0)
        thr_row_kernel<<<ceil_div(n_thr, 256), 256, 0, st>>>(A->n_rows, n_thr, kSegP, c.row_ptr, c.thr_row);
    GKO_TRY(seg_alloc(&c.seg, A->nnz, kSegP));
    int32_t* d_stats;
    GKO_TRY(dev_alloc(&d_stats, 2));
    GKO_CUDA(cudaMemsetAsync(d_stats, 0, 2 * sizeof(int32_t), st));
    if (A->n_rows > 0) {
        const int grid = std::min(ceil_div(A->n_rows, 256), 152 * 8);
        row_stats_kernel<<<grid, 256, 0, st>>>(A->n_rows, c.row_ptr, c.col, d_stats);
    }
    int32_t h[2];
    GKO_CUDA(cudaMemcpyAsync(h, d_stats, sizeof(h), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    cudaFree(d_stats);
    GKO_CUDA(cudaGetLastError());
    c.max_len = h[0];
    c.band = h[1];
    c.mean_len = A->n_rows ? static_cast<double>(A->nnz) / A->n_rows : 0.0;
    return GKO_OK;
}

// ------------------------------------------------------------ y = beta*y

__global__ void scale_kernel(int64_t n, double* __restrict__ y, double beta)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        y[i] = beta == 0.0 ? 0.0 : beta * y[i];
}

int scale_vector(int64_t n, double* y, double beta, cudaStream_t st)
{
    if (n <= 0) return GKO_OK;
    scale_kernel<<<std::min(ceil_div(n, 256), 152 * 8), 256, 0, st>>>(n, y, beta);
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

// ----------------------------------------------- classical subwarp per row

template <int SW, bool kAlpha, bool kBeta>
__global__ void __launch_bounds__(256)
    csr_subwarp_kernel(int64_t n_rows, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                       double alpha, double beta)
{
    using G = subwarp<SW>;
    constexpr int kRowsPerWarp = kWarp / SW;
    const int lane = G::rank();
    const int sub = (threadIdx.x % kWarp) / SW;
    const int64_t warp = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) / kWarp;
    const int64_t n_warps = static_cast<int64_t>(gridDim.x) * blockDim.x / kWarp;
    // warp-uniform loop: every lane reaches the shuffles together
    for (int64_t base = warp * kRowsPerWarp; base < n_rows; base += n_warps * kRowsPerWarp) {
        const int64_t r = base + sub;
        double acc = 0.0;
        if (r < n_rows) {
            const int32_t k1 = row_ptr[r + 1];
            for (int32_t k = row_ptr[r] + lane; k < k1; k += SW) acc = fma(val[k], ldg(x + col[k]), acc);
        }
        acc = G::reduce_sum(acc);
        if (r < n_rows && lane == 0) seg_store<kAlpha, kBeta>(y, r, acc, alpha, beta);
    }
}

template <int SW>
static void launch_subwarp(const gko_matrix* A, const double* x, double* y, double alpha, double beta,
                           cudaStream_t st)
{
    const CsrPart& c = A->csr;
    const int64_t rows_per_block = 256 / SW;  // grid-stride beyond 16 CTAs per SM
    const int grid = static_cast<int>(std::min<int64_t>((A->n_rows + rows_per_block - 1) / rows_per_block,
                                                        152LL * 16));
    const bool a = alpha != 1.0, b = beta != 0.0;
#define GKO_SW_LAUNCH(KA, KB)                                                                           \
    csr_subwarp_kernel<SW, KA, KB><<<grid, 256, 0, st>>>(A->n_rows, c.row_ptr, c.col, c.val, x, y, alpha, \
                                                         beta)
    if (a && b)
        GKO_SW_LAUNCH(true, true);
    else if (a)
        GKO_SW_LAUNCH(true, false);
    else if (b)
        GKO_SW_LAUNCH(false, true);
    else
        GKO_SW_LAUNCH(false, false);
#undef GKO_SW_LAUNCH
}

// --------------------------------------------------- load-balanced launch

static SegScratch scratch_of(const SegArrays& sa)
{
    return SegScratch{sa.tail_val, sa.tail_row, sa.tail_pass, sa.head_val, sa.head_row};
}

int launch_seg(int64_t n_rows, int64_t nnz, const int32_t* row_ptr, const int32_t* rows, const int32_t* col,
               const double* val, const int32_t* thr_row, const SegArrays& sa, const double* x, double* y,
               double alpha, double beta, uint32_t* err, bool coo, cudaStream_t st, bool accumulate)
{
    const SegScratch sc = scratch_of(sa);
    cudaError_t e;
    if (accumulate) {  // y += alpha * A x, rows without entries untouched
        if (nnz == 0) return GKO_OK;
        if (alpha != 1.0)
            e = seg_launch<kSegPCoo, double, double, true, true, true, true>(n_rows, nnz, row_ptr, rows, col, val,
                                                                         thr_row, sc, x, y, alpha, 1.0, err, st);
        else
            e = seg_launch<kSegPCoo, double, double, false, true, true, true>(n_rows, nnz, row_ptr, rows, col, val,
                                                                          thr_row, sc, x, y, alpha, 1.0, err, st);
        if (e != cudaSuccess) return cuda_fail(e, "load-balanced SpMV launch");
        return GKO_OK;
    }
    if (nnz == 0) return scale_vector(n_rows, y, beta, st);
    const bool a = alpha != 1.0, b = beta != 0.0;
#define GKO_SEG(KA, KB)                                                                                          \
    e = coo ? seg_launch<kSegPCoo, double, double, KA, KB, true, false>(n_rows, nnz, row_ptr, rows, col, val,       \
                                                                     thr_row, sc, x, y, alpha, beta, err, st)    \
            : seg_launch<kSegP, double, double, KA, KB, false, false>(n_rows, nnz, row_ptr, rows, col, val,      \
                                                                      thr_row, sc, x, y, alpha, beta, err, st)
    if (a && b)
        GKO_SEG(true, true);
    else if (a)
        GKO_SEG(true, false);
    else if (b)
        GKO_SEG(false, true);
    else
        GKO_SEG(false, false);
#undef GKO_SEG
    if (e != cudaSuccess) return cuda_fail(e, "load-balanced SpMV launch");
    return GKO_OK;
}

// ------------------------------------------------------------- dispatch

int spmv_csr(const gko_matrix* A, int config, const double* x, double* y, double alpha, double beta,
             cudaStream_t st)
{
    if (A->n_rows == 0) return GKO_OK;
    if (A->nnz == 0) return scale_vector(A->n_rows, y, beta, st);
    switch (config) {
        case GKO_CFG_CSR_SUBWARP_1: launch_subwarp<1>(A, x, y, alpha, beta, st); break;
        case GKO_CFG_CSR_SUBWARP_2: launch_subwarp<2>(A, x, y, alpha, beta, st); break;
        case GKO_CFG_CSR_SUBWARP_4: launch_subwarp<4>(A, x, y, alpha, beta, st); break;
        case GKO_CFG_CSR_SUBWARP_8: launch_subwarp<8>(A, x, y, alpha, beta, st); break;
        case GKO_CFG_CSR_SUBWARP_16: launch_subwarp<16>(A, x, y, alpha, beta, st); break;
        case GKO_CFG_CSR_SUBWARP_32: launch_subwarp<32>(A, x, y, alpha, beta, st); break;
        case GKO_CFG_CSR_ROWBLOCK: return spmv_csr_rowblock(A, x, y, alpha, beta, st);
        case GKO_CFG_CSR_BANDED: return spmv_csr_banded(A, x, y, alpha, beta, st);
        case GKO_CFG_DEFAULT:
            if (rowblock_preferred(A)) return spmv_csr_rowblock(A, x, y, alpha, beta, st);
            [[fallthrough]];
        case GKO_CFG_CSR_NNZSPLIT:
            return launch_seg(A->n_rows, A->nnz, A->csr.row_ptr, nullptr, A->csr.col, A->csr.val, A->csr.thr_row,
                              A->csr.seg, x, y, alpha, beta, A->d_err, false, st, false);
        default: return fail(GKO_ERR_INVALID_ARG, "configuration does not apply to CSR");
    }
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

int spmv_coo(const gko_matrix* A, const CooPart& coo, const double* x, double* y, double alpha, double beta,
             cudaStream_t st)
{
    if (A->n_rows == 0) return GKO_OK;
    return launch_seg(A->n_rows, coo.nnz, nullptr, coo.row, coo.col, coo.val, nullptr, coo.seg, x, y, alpha, beta,
                      A->d_err, true, st, false);
}

}  // namespace gko
