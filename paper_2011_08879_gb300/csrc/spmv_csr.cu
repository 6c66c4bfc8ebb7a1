// CSR SpMV (paper Sec. 6.1: y = A x in CSR, bounded by 12 bytes/entry):
//  * classical subwarp-per-row kernel (subwarp of 1..32 lanes, chosen at
//    run time; the paper's cooperative-group subwarps and Listing 2's
//    butterfly reduction);
//  * load-balanced equal-nnz kernel (segmented.cuh);
//  * binned kernel: rows grouped by length, each group by subwarps sized to
//    it (the default for skewed rows);
//  * banded kernel: the x window of a row block staged in shared memory.
#include <algorithm>
#include <utility>
#include <vector>

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

// Row-length bins of the binned kernel: bin b holds the rows whose length
// lies in (kBinMax[b-1], kBinMax[b]]; the last bin is unbounded.
__host__ __device__ __forceinline__ int csr_bin(int32_t len)
{
    return len <= 8 ? 0 : len <= 20 ? 1 : len <= 48 ? 2 : len <= 128 ? 3 : len <= 512 ? 4 : 5;
}

__global__ void bin_flag_kernel(int64_t n_rows, const int32_t* __restrict__ row_ptr, int b,
                                int64_t* __restrict__ flag)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r < n_rows) flag[r] = csr_bin(row_ptr[r + 1] - row_ptr[r]) == b;
}

// stable scatter: rows of bin b in ascending order at out[off[r]]
__global__ void bin_scatter_kernel(int64_t n_rows, const int32_t* __restrict__ row_ptr, int b,
                                   const int64_t* __restrict__ off, int32_t* __restrict__ out)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r < n_rows && csr_bin(row_ptr[r + 1] - row_ptr[r]) == b) out[off[r]] = static_cast<int32_t>(r);
}

// Rows per task of the one-launch binned kernel, by bin: four passes of a
// 256-thread CTA over subwarps of 1, 2, 4, 8, 32 lanes; one long row per
// task in the last bin.
constexpr int kBinSW[kCsrBins] = {1, 2, 4, 8, 32, 0};
constexpr int kTaskPasses = 4;
static int bin_task_rows(int b) { return kBinSW[b] ? 256 / kBinSW[b] * kTaskPasses : 1; }

// Tasks of the one-launch binned kernel: chunks of bin_rows (a bin's rows,
// bin_task_rows(b) at a time) ordered by their first row, so the CTAs that
// run together work on neighbouring rows whatever their bins (their
// matrix sectors and x stay in L2 between them).  One int4 per task:
// (start in bin_rows, row count, bin, 0).
static int csr_build_bin_tasks(gko_matrix* A, cudaStream_t st)
{
    CsrPart& c = A->csr;
    dev_free(c.bin_tasks);
    c.n_bin_tasks = 0;
    const int64_t n = A->n_rows;
    if (n == 0) return GKO_OK;
    std::vector<int32_t> rows(static_cast<size_t>(n));
    GKO_CUDA(cudaMemcpyAsync(rows.data(), c.bin_rows, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    std::vector<std::pair<int32_t, int4>> t;
    for (int b = 0; b < kCsrBins; ++b) {
        const int64_t per = bin_task_rows(b);
        for (int64_t q = c.bin_off[b]; q < c.bin_off[b + 1]; q += per) {
            const int64_t cnt = std::min<int64_t>(per, c.bin_off[b + 1] - q);
            t.push_back({rows[q], make_int4(static_cast<int>(q), static_cast<int>(cnt), b, 0)});
        }
    }
    std::stable_sort(t.begin(), t.end(), [](const std::pair<int32_t, int4>& a, const std::pair<int32_t, int4>& b) {
        return a.first < b.first;
    });
    std::vector<int4> h(t.size());
    for (size_t i = 0; i < t.size(); ++i) h[i] = t[i].second;
    GKO_TRY(dev_alloc(&c.bin_tasks, static_cast<int64_t>(h.size())));
    GKO_CUDA(cudaMemcpyAsync(c.bin_tasks, h.data(), h.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    c.n_bin_tasks = static_cast<int64_t>(h.size());
    return GKO_OK;
}

// Build bin_rows (the rows grouped by bin, ascending inside each bin), the
// bin offsets and the task list.  Synchronises the stream.
static int csr_build_bins(gko_matrix* A, cudaStream_t st)
{
    CsrPart& c = A->csr;
    const int64_t n = A->n_rows;
    dev_free(c.bin_rows);
    for (int b = 0; b <= kCsrBins; ++b) c.bin_off[b] = 0;
    if (n == 0) return GKO_OK;
    GKO_TRY(dev_alloc(&c.bin_rows, n));
    int64_t *flag, *off;
    GKO_TRY(dev_alloc(&flag, n));
    if (dev_alloc(&off, n + 1) != GKO_OK) {
        cudaFree(flag);
        return GKO_ERR_OUT_OF_MEMORY;
    }
    int s = GKO_OK;
    int64_t base = 0;
    for (int b = 0; b < kCsrBins && s == GKO_OK; ++b) {
        bin_flag_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, c.row_ptr, b, flag);
        s = exclusive_scan(flag, off, n, st);
        if (s != GKO_OK) break;
        bin_scatter_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, c.row_ptr, b, off, c.bin_rows + base);
        int64_t cnt = 0;
        cudaError_t e = cudaMemcpyAsync(&cnt, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "row binning");
        c.bin_off[b] = base;
        base += cnt;
        c.bin_off[b + 1] = base;
    }
    cudaFree(flag);
    cudaFree(off);
    if (s == GKO_OK) GKO_CUDA(cudaGetLastError());
    if (s == GKO_OK) s = csr_build_bin_tasks(A, st);
    return s;
}

int seg_alloc(SegArrays* s, int64_t nnz, int P, int threads)
{
    seg_free(s);
    const int64_t tile = static_cast<int64_t>(threads) * P;
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
    GKO_TRY(seg_alloc(&c.seg, A->nnz, kSegP, kSegThreads));
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
    return csr_build_bins(A, st);
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

// ------------------------------------------------- binned rows (skewed)

// Four entries of one lane: indices and values of entries k, k + S, k + 2S,
// k + 3S (those below k1) are loaded first, then the four gathers are
// issued, then two FMA chains.  With x gathered at random from L2 (skewed,
// unstructured matrices) each lane thus keeps four gathers in flight
// instead of one per memory round trip.
template <int S, bool kL2 = false>
__device__ __forceinline__ void fma4(int32_t k, int32_t k1, const int32_t* __restrict__ col,
                                     const double* __restrict__ val, const double* __restrict__ x, double& a0,
                                     double& a1)
{
    int32_t c[4];
    double v[4], xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int32_t kk = k + u * S;
        c[u] = kk < k1 ? col[kk] : -1;
        v[u] = kk < k1 ? val[kk] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = c[u] >= 0 ? (kL2 ? __ldcg(x + c[u]) : ldg(x + c[u])) : 0.0;
    if (c[0] >= 0) a0 = fma(v[0], xv[0], a0);
    if (c[1] >= 0) a1 = fma(v[1], xv[1], a1);
    if (c[2] >= 0) a0 = fma(v[2], xv[2], a0);
    if (c[3] >= 0) a1 = fma(v[3], xv[3], a1);
}

// One CTA per task: the task's rows of one bin, by subwarps of SW lanes
// (warp w of the CTA takes row groups w, w + 8, ...), four entries per lane
// in flight (fma4).  On matrices whose columns are spread at random
// (power-law rows over 2M columns) every gather is a separate 32-byte L2
// sector; GB300 serves such gathers at ~270 G/s (one per SM clock), which
// bounds those products, not HBM bandwidth.
template <int SW, bool kAlpha, bool kBeta, bool kL2>
__device__ __forceinline__ void task_rows(const int32_t* __restrict__ rows, int count,
                                          const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                          const double* __restrict__ val, const double* __restrict__ x,
                                          double* __restrict__ y, double alpha, double beta)
{
    using G = subwarp<SW>;
    constexpr int kRowsPerWarp = kWarp / SW;
    const int lane = G::rank();
    const int sub = (threadIdx.x % kWarp) / SW;
    const int w = threadIdx.x / kWarp;
    for (int base = w * kRowsPerWarp; base < count; base += (256 / kWarp) * kRowsPerWarp) {
        const int q = base + sub;
        const int32_t r = q < count ? rows[q] : 0;
        double a0 = 0.0, a1 = 0.0;
        if (q < count) {
            const int32_t k1 = row_ptr[r + 1];
            for (int32_t k = row_ptr[r] + lane; k < k1; k += 4 * SW) fma4<SW, kL2>(k, k1, col, val, x, a0, a1);
        }
        const double acc = G::reduce_sum(a0 + a1);
        if (q < count && lane == 0) seg_store<kAlpha, kBeta>(y, r, acc, alpha, beta);
    }
}

// kL2: gathers of x through L2 only (ld.global.cg), for matrices whose
// columns are spread over the whole vector: L1 would rarely reuse them
template <bool kAlpha, bool kBeta, bool kL2>
__global__ void __launch_bounds__(256)
    csr_binned_kernel(const int4* __restrict__ tasks, const int32_t* __restrict__ bin_rows,
                      const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                      const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                      double alpha, double beta)
{
    __shared__ double sh[8];
    const int4 t = tasks[blockIdx.x];
    const int32_t* rows = bin_rows + t.x;
    switch (t.z) {
        case 0: task_rows<1, kAlpha, kBeta, kL2>(rows, t.y, row_ptr, col, val, x, y, alpha, beta); break;
        case 1: task_rows<2, kAlpha, kBeta, kL2>(rows, t.y, row_ptr, col, val, x, y, alpha, beta); break;
        case 2: task_rows<4, kAlpha, kBeta, kL2>(rows, t.y, row_ptr, col, val, x, y, alpha, beta); break;
        case 3: task_rows<8, kAlpha, kBeta, kL2>(rows, t.y, row_ptr, col, val, x, y, alpha, beta); break;
        case 4: task_rows<32, kAlpha, kBeta, kL2>(rows, t.y, row_ptr, col, val, x, y, alpha, beta); break;
        default: {  // one long row, the whole CTA
            const int32_t r = rows[0];
            const int32_t k0 = row_ptr[r], k1 = row_ptr[r + 1];
            double a0 = 0.0, a1 = 0.0;
            for (int32_t k = k0 + static_cast<int32_t>(threadIdx.x); k < k1; k += 1024)
                fma4<256, kL2>(k, k1, col, val, x, a0, a1);
            const double s = subwarp<32>::reduce_sum(a0 + a1);
            if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int w = 0; w < 8; ++w) tot += sh[w];
                seg_store<kAlpha, kBeta>(y, r, tot, alpha, beta);
            }
        }
    }
}

// Binned CSR SpMV: every row is computed once by the kernel of its length
// bin (1, 2, 4, 8 or 32 lanes per row, or a whole CTA for rows longer than
// 512), so rows of any length mix take full occupancy, each entry one FMA,
// and no partial sums cross threads except the lanes of one row.  All bins
// go in one launch (csr_binned_kernel over the task list, in row order).
static void launch_binned(const gko_matrix* A, const double* x, double* y, double alpha, double beta,
                          cudaStream_t st)
{
    const CsrPart& c = A->csr;
    const bool a = alpha != 1.0, b = beta != 0.0;
    if (c.n_bin_tasks > 0) {  // tasks <= rows < 2^31
        const unsigned g = static_cast<unsigned>(c.n_bin_tasks);
        const bool l2 = coo_entries_per_thread(A) == kSegPCoo;  // scattered columns (the COO kernel's test)
#define GKO_BT(KA, KB)                                                                                                  \
    (l2 ? csr_binned_kernel<KA, KB, true><<<g, 256, 0, st>>>(c.bin_tasks, c.bin_rows, c.row_ptr, c.col, c.val, x, y, \
                                                              alpha, beta)                                              \
        : csr_binned_kernel<KA, KB, false><<<g, 256, 0, st>>>(c.bin_tasks, c.bin_rows, c.row_ptr, c.col, c.val, x, y, \
                                                               alpha, beta))
        if (a && b)
            GKO_BT(true, true);
        else if (a)
            GKO_BT(true, false);
        else if (b)
            GKO_BT(false, true);
        else
            GKO_BT(false, false);
#undef GKO_BT
        return;
    }
    scale_vector(A->n_rows, y, beta, st);  // no rows (n = 0): only the beta scaling
}

// --------------------------------------------------- load-balanced launch

static SegScratch scratch_of(const SegArrays& sa)
{
    return SegScratch{sa.tail_val, sa.tail_row, sa.tail_pass, sa.head_val, sa.head_row};
}

int coo_entries_per_thread(const gko_matrix* A)
{
    const int64_t band = A->csr.band;
    return (band >= 0 && band <= std::max<int64_t>(4096, A->n_rows / 16)) ? kSegPCooLocal : kSegPCoo;
}

template <int PC>
static cudaError_t launch_coo_p(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* rows, const int32_t* col,
                                const double* val, const SegScratch& sc, const double* x, double* y, double alpha,
                                double beta, uint32_t* err, cudaStream_t st, bool accumulate)
{
    const bool a = alpha != 1.0, b = beta != 0.0;
    // matrices with scattered columns (the smaller tiles) gather x through L2 only
    constexpr bool kL2 = PC == kSegPCoo;
    if (accumulate)  // y += alpha * A x, rows without entries untouched
        return a ? seg_launch<PC, double, double, true, true, true, true, false, kSegThreadsCoo, kL2>(
                       n_rows, n_cols, nnz, nullptr, rows, col, val, nullptr, sc, x, y, alpha, 1.0, err, st)
                 : seg_launch<PC, double, double, false, true, true, true, false, kSegThreadsCoo, kL2>(
                       n_rows, n_cols, nnz, nullptr, rows, col, val, nullptr, sc, x, y, alpha, 1.0, err, st);
#define GKO_COO(KA, KB)                                                                                   \
    return seg_launch<PC, double, double, KA, KB, true, false, false, kSegThreadsCoo, kL2>(               \
        n_rows, n_cols, nnz, nullptr, rows, col, val, nullptr, sc, x, y, alpha, beta, err, st)
    if (a && b) GKO_COO(true, true);
    if (a) GKO_COO(true, false);
    if (b) GKO_COO(false, true);
    GKO_COO(false, false);
#undef GKO_COO
}

int launch_seg(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row_ptr, const int32_t* rows, const int32_t* col,
               const double* val, const int32_t* thr_row, const SegArrays& sa, const double* x, double* y,
               double alpha, double beta, uint32_t* err, bool coo, cudaStream_t st, bool accumulate, int coo_p)
{
    const SegScratch sc = scratch_of(sa);
    cudaError_t e;
    if (accumulate && nnz == 0) return GKO_OK;
    if (!accumulate && nnz == 0) return scale_vector(n_rows, y, beta, st);
    if (coo) {
        e = coo_p == kSegPCooLocal
                ? launch_coo_p<kSegPCooLocal>(n_rows, n_cols, nnz, rows, col, val, sc, x, y, alpha, beta, err, st,
                                              accumulate)
                : launch_coo_p<kSegPCoo>(n_rows, n_cols, nnz, rows, col, val, sc, x, y, alpha, beta, err, st,
                                         accumulate);
        if (e != cudaSuccess) return cuda_fail(e, "load-balanced COO SpMV launch");
        return GKO_OK;
    }
    const bool a = alpha != 1.0, b = beta != 0.0;
#define GKO_SEG(KA, KB)                                                                                          \
    e = seg_launch<kSegP, double, double, KA, KB, false, false>(n_rows, n_cols, nnz, row_ptr, rows, col, val,    \
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

// Kernel behind GKO_CFG_DEFAULT, from the row-length statistics, as measured
// on GB300 (FP64, L2 flushed): rows of close length (max <= 2 mean + 16) go
// one thread per row with direct loads when at most 8 long (7-point 160^3:
// 73 % of HBM bandwidth vs 61 % for the staged row blocks), staged row blocks
// up to 20 (random banded, 16 per row: 69 %), four lanes per row beyond
// (27-point 128^3: 69 % vs 58 %); skewed rows take the row-length bins
// (power-law 2M rows, mean 20, max 20k: 229 us vs 439 us for the equal-nnz
// split; random gathers of x bound that matrix, see task_rows).
int default_csr_config(const gko_matrix* A)
{
    if (!rowblock_preferred(A)) return GKO_CFG_CSR_BINNED;
    if (A->csr.max_len <= 8) return GKO_CFG_CSR_SUBWARP_1;
    if (A->csr.max_len <= 20) return GKO_CFG_CSR_ROWBLOCK;
    return GKO_CFG_CSR_SUBWARP_4;
}

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
        case GKO_CFG_CSR_BINNED: launch_binned(A, x, y, alpha, beta, st); break;
        case GKO_CFG_DEFAULT:
            switch (default_csr_config(A)) {
                case GKO_CFG_CSR_SUBWARP_1: launch_subwarp<1>(A, x, y, alpha, beta, st); break;
                case GKO_CFG_CSR_SUBWARP_4: launch_subwarp<4>(A, x, y, alpha, beta, st); break;
                case GKO_CFG_CSR_ROWBLOCK: return spmv_csr_rowblock(A, x, y, alpha, beta, st);
                default: launch_binned(A, x, y, alpha, beta, st); break;
            }
            break;
        case GKO_CFG_CSR_NNZSPLIT:
            return launch_seg(A->n_rows, A->n_cols, A->nnz, A->csr.row_ptr, nullptr, A->csr.col, A->csr.val, A->csr.thr_row,
                              A->csr.seg, x, y, alpha, beta, A->d_err, false, st, false, 0);
        default: return fail(GKO_ERR_INVALID_ARG, "configuration does not apply to CSR");
    }
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

int spmv_coo(const gko_matrix* A, const CooPart& coo, const double* x, double* y, double alpha, double beta,
             cudaStream_t st)
{
    if (A->n_rows == 0) return GKO_OK;
    return launch_seg(A->n_rows, A->n_cols, coo.nnz, nullptr, coo.row, coo.col, coo.val, nullptr, coo.seg, x, y, alpha, beta,
                      A->d_err, true, st, false, coo.P);
}

}  // namespace gko
