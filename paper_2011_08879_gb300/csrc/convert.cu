// Format conversions on the device.  Every conversion moves indices and
// values bit for bit (no floating-point arithmetic); padding follows the
// format definitions of the public header.  Work is split by stored entries
// with the CSR analysis (thr_row: the row holding entry g*P), so rows of any
// length cost the same; row lengths are turned into offsets by an exclusive
// scan.  Sizes are read back to the host, so conversions synchronise.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace gko {

// --------------------------------------------------------------- scan

constexpr int kScanBlock = 1024;

// per block of kScanBlock elements: inclusive block sum
__global__ void scan_reduce_kernel(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ sums)
{
    __shared__ int64_t sh[32];
    const int64_t i = blockIdx.x * static_cast<int64_t>(kScanBlock) + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = sh[threadIdx.x];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

// block-local exclusive scan plus the block's offset
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* sh, int64_t* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t s = lane < (blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        sh[lane] = s;  // inclusive warp prefix
    }
    __syncthreads();
    const int64_t warp_off = w > 0 ? sh[w - 1] : 0;
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    return warp_off + inc - v;
}

// exclusive scan of the block sums, one block, any length (sequential chunks)
__global__ void scan_sums_kernel(int64_t* __restrict__ sums, int64_t nb)
{
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < nb ? sums[i] : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_scan(v, sh, &tot);
        __syncthreads();
        if (i < nb) sums[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
}

__global__ void scan_final_kernel(const int64_t* __restrict__ in, int64_t n, const int64_t* __restrict__ offs,
                                  int64_t* __restrict__ out)
{
    __shared__ int64_t sh[32];
    const int64_t i = blockIdx.x * static_cast<int64_t>(kScanBlock) + threadIdx.x;
    const int64_t v = i < n ? in[i] : 0;
    const int64_t ex = block_exclusive_scan(v, sh, nullptr);
    if (i <= n) out[i] = offs[blockIdx.x] + ex;  // out has n + 1 entries; out[n] = total
}

// out[0..n] = exclusive scan of in[0..n-1] (out[n] = total).  Temporary
// block sums are allocated stream-ordered.
int exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st)
{
    const int64_t nb = n / kScanBlock + 1;  // +1 block so that out[n] is written
    int64_t* sums = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&sums), nb * sizeof(int64_t), st));
    scan_reduce_kernel<<<static_cast<unsigned>(nb), kScanBlock, 0, st>>>(in, n, sums);
    scan_sums_kernel<<<1, kScanBlock, 0, st>>>(sums, nb);
    scan_final_kernel<<<static_cast<unsigned>(nb), kScanBlock, 0, st>>>(in, n, sums, out);
    GKO_CUDA(cudaFreeAsync(sums, st));
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

// ------------------------------------------------------------ helpers

template <typename T>
static int read_back(T* host, const T* dev, cudaStream_t st)
{
    GKO_CUDA(cudaMemcpyAsync(host, dev, sizeof(T), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    return GKO_OK;
}

// Walk the entries [g*P, g*P+P) of a CSR matrix with their row r and slot
// j = k - row_ptr[r]; F(k, r, j) is called for each.
template <typename F>
__device__ __forceinline__ void for_entries(int64_t g, int64_t P, int64_t nnz, int64_t n_rows,
                                            const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ thr_row,
                                            F f)
{
    const int64_t s = g * P;
    if (s >= nnz) return;
    const int64_t e = min(s + P, nnz);
    int64_t r = thr_row[g];
    int64_t start = row_ptr[r], end = row_ptr[r + 1];
    for (int64_t k = s; k < e; ++k) {
        while (k >= end) {
            ++r;
            start = end;
            end = row_ptr[r + 1];
        }
        f(k, r, k - start);
    }
    (void)n_rows;
}

// ------------------------------------------------------------ CSR <-> COO

__global__ void csr_rows_kernel(int64_t nnz, int64_t n_rows, const int32_t* __restrict__ row_ptr,
                                const int32_t* __restrict__ thr_row, int32_t* __restrict__ row)
{
    const int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    for_entries(g, kSegP, nnz, n_rows, row_ptr, thr_row,
                [&](int64_t k, int64_t r, int64_t) { row[k] = static_cast<int32_t>(r); });
}

int convert_csr_to_coo(gko_matrix* A, cudaStream_t st)
{
    free_format(A, GKO_FMT_COO);
    CooPart& c = A->coo;
    const int64_t alloc = padded_len(A->nnz);
    GKO_TRY(dev_alloc(&c.row, alloc));
    GKO_TRY(dev_alloc(&c.col, alloc));
    GKO_TRY(dev_alloc(&c.val, alloc));
    GKO_CUDA(cudaMemsetAsync(c.row, 0, alloc * sizeof(int32_t), st));
    GKO_CUDA(cudaMemcpyAsync(c.col, A->csr.col, alloc * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    GKO_CUDA(cudaMemcpyAsync(c.val, A->csr.val, alloc * sizeof(double), cudaMemcpyDeviceToDevice, st));
    const int64_t n_thr = (A->nnz + kSegP - 1) / kSegP;
    if (n_thr > 0)
        csr_rows_kernel<<<ceil_div(n_thr, 256), 256, 0, st>>>(A->nnz, A->n_rows, A->csr.row_ptr, A->csr.thr_row,
                                                               c.row);
    c.nnz = A->nnz;
    c.P = coo_entries_per_thread(A);
    GKO_TRY(seg_alloc(&c.seg, c.nnz, c.P, kSegThreadsCoo));
    GKO_CUDA(cudaGetLastError());
    GKO_CUDA(cudaStreamSynchronize(st));
    A->has[GKO_FMT_COO] = true;
    return GKO_OK;
}

// row_ptr[r] = number of entries with row < r (rows sorted), r = 0..n
__global__ void coo_row_ptr_kernel(int64_t n_rows, int64_t nnz, const int32_t* __restrict__ row,
                                   int32_t* __restrict__ row_ptr)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r > n_rows) return;
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (row[mid] < r)
            lo = mid + 1;
        else
            hi = mid;
    }
    row_ptr[r] = static_cast<int32_t>(lo);
}

static int alloc_csr(gko_matrix* A)
{
    CsrPart& c = A->csr;
    const int64_t alloc = padded_len(A->nnz);
    GKO_TRY(dev_alloc(&c.row_ptr, padded_len(A->n_rows + 1)));
    GKO_TRY(dev_alloc(&c.col, alloc));
    GKO_TRY(dev_alloc(&c.val, alloc));
    return GKO_OK;
}

static int finish_csr(gko_matrix* A, cudaStream_t st)
{
    const int64_t alloc = padded_len(A->nnz);
    // zero the pads past nnz and n+1 (bulk copies read whole 16-byte groups)
    const int64_t rp_alloc = padded_len(A->n_rows + 1);
    GKO_CUDA(cudaMemsetAsync(A->csr.row_ptr + A->n_rows + 1, 0, (rp_alloc - A->n_rows - 1) * sizeof(int32_t), st));
    GKO_CUDA(cudaMemsetAsync(A->csr.col + A->nnz, 0, (alloc - A->nnz) * sizeof(int32_t), st));
    GKO_CUDA(cudaMemsetAsync(A->csr.val + A->nnz, 0, (alloc - A->nnz) * sizeof(double), st));
    GKO_TRY(csr_analyse(A, st));
    A->has[GKO_FMT_CSR] = true;
    return GKO_OK;
}

int convert_coo_to_csr(gko_matrix* A, cudaStream_t st)
{
    free_format(A, GKO_FMT_CSR);
    GKO_TRY(alloc_csr(A));
    const CooPart& c = A->coo;
    coo_row_ptr_kernel<<<ceil_div(A->n_rows + 1, 256), 256, 0, st>>>(A->n_rows, c.nnz, c.row, A->csr.row_ptr);
    GKO_CUDA(cudaMemcpyAsync(A->csr.col, c.col, c.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    GKO_CUDA(cudaMemcpyAsync(A->csr.val, c.val, c.nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
    GKO_CUDA(cudaGetLastError());
    return finish_csr(A, st);
}

// ------------------------------------------------------------ CSR <-> ELL


// Row r of an ELL part of width K: slot k (column-major, k*n_pad + r) gets
// the row's k-th entry, or padding (col -1, val +0.0) when k >= its length.
// One thread per row: the writes of consecutive threads are contiguous, and
// the padding is written in the same pass.
__global__ void csr_to_ell_rows_kernel(int64_t n_rows, int64_t n_pad, int64_t K, const int32_t* __restrict__ row_ptr,
                                       const int32_t* __restrict__ col, const double* __restrict__ val,
                                       int32_t* __restrict__ ecol, double* __restrict__ eval)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= n_pad) return;
    int64_t a = 0, L = 0;
    if (r < n_rows) {
        a = row_ptr[r];
        L = row_ptr[r + 1] - a;
    }
    for (int64_t k = 0; k < K; ++k) {
        if (k < L) {
            ecol[k * n_pad + r] = col[a + k];
            eval[k * n_pad + r] = val[a + k];
        } else {
            ecol[k * n_pad + r] = -1;
            eval[k * n_pad + r] = 0.0;
        }
    }
}

int ell_fill(gko_matrix* A, EllPart* e, int64_t K, cudaStream_t st)
{
    e->K = K;
    e->n_pad = (A->n_rows + 31) / 32 * 32;
    const int64_t slots = e->K * e->n_pad;
    const int64_t alloc = padded_len(slots);
    GKO_TRY(dev_alloc(&e->col, alloc));
    GKO_TRY(dev_alloc(&e->val, alloc));
    // the allocation tail past the slots is zero (bulk copies may read it)
    GKO_CUDA(cudaMemsetAsync(e->col + slots, 0, (alloc - slots) * sizeof(int32_t), st));
    GKO_CUDA(cudaMemsetAsync(e->val + slots, 0, (alloc - slots) * sizeof(double), st));
    if (K > 0 && e->n_pad > 0)
        csr_to_ell_rows_kernel<<<ceil_div(e->n_pad, 256), 256, 0, st>>>(A->n_rows, e->n_pad, K, A->csr.row_ptr,
                                                                         A->csr.col, A->csr.val, e->col, e->val);
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

int convert_csr_to_ell(gko_matrix* A, cudaStream_t st)
{
    const int64_t K = A->csr.max_len;
    const int64_t n_pad = (A->n_rows + 31) / 32 * 32;
    const double limit = std::max(A->ell_factor * static_cast<double>(A->nnz), static_cast<double>(1 << 22));
    if (static_cast<double>(K) * static_cast<double>(n_pad) > limit)
        return fail(GKO_ERR_FORMAT_TOO_LARGE, "ELL padding exceeds the size limit (K * n_pad > max(factor * nnz, 2^22))");
    free_format(A, GKO_FMT_ELL);
    GKO_TRY(ell_fill(A, &A->ell, K, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    A->has[GKO_FMT_ELL] = true;
    return GKO_OK;
}

// per-row count of stored (non-padding) ELL slots
__global__ void ell_count_kernel(int64_t n_rows, int64_t n_pad, int64_t K, const int32_t* __restrict__ ecol,
                                 int64_t* __restrict__ cnt, int add)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= n_rows) return;
    int64_t c = 0;
    for (int64_t k = 0; k < K; ++k) c += ecol[k * n_pad + r] >= 0;
    cnt[r] = add ? cnt[r] + c : c;
}

// gather stored ELL slots of row r (slot order) to out[off[r] ...]; returns via count
__global__ void ell_gather_kernel(int64_t n_rows, int64_t n_pad, int64_t K, const int32_t* __restrict__ ecol,
                                  const double* __restrict__ eval, const int64_t* __restrict__ off,
                                  int32_t* __restrict__ col, double* __restrict__ val)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= n_rows) return;
    int64_t o = off[r];
    for (int64_t k = 0; k < K; ++k) {
        const int32_t c = ecol[k * n_pad + r];
        if (c < 0) continue;
        col[o] = c;
        val[o] = eval[k * n_pad + r];
        ++o;
    }
}

__global__ void offsets_to_row_ptr_kernel(int64_t n, const int64_t* __restrict__ off, int32_t* __restrict__ rp,
                                          uint32_t* err)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i > n) return;
    const int64_t v = off[i];
    if (v > INT32_MAX) raise_error(err, kErrOverflow);
    rp[i] = static_cast<int32_t>(v);
}

// counts (int64, n) -> CSR row_ptr (and the int64 offsets, kept for gathers)
static int counts_to_csr(gko_matrix* A, int64_t* cnt, int64_t** off_out, cudaStream_t st)
{
    int64_t* off = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&off), (A->n_rows + 1) * sizeof(int64_t), st));
    GKO_TRY(exclusive_scan(cnt, off, A->n_rows, st));
    int64_t total = 0;
    GKO_TRY(read_back(&total, off + A->n_rows, st));
    if (total != A->nnz) {
        cudaFreeAsync(off, st);
        return fail(GKO_ERR_INVALID_MATRIX, "stored entries of the source format disagree with nnz");
    }
    GKO_TRY(alloc_csr(A));
    offsets_to_row_ptr_kernel<<<ceil_div(A->n_rows + 1, 256), 256, 0, st>>>(A->n_rows, off, A->csr.row_ptr,
                                                                            A->d_err);
    *off_out = off;
    return GKO_OK;
}

int convert_ell_to_csr(gko_matrix* A, cudaStream_t st)
{
    free_format(A, GKO_FMT_CSR);
    const EllPart& e = A->ell;
    int64_t* cnt = nullptr;
    int64_t* off = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&cnt), (A->n_rows + 1) * sizeof(int64_t), st));
    const int grid = ceil_div(std::max<int64_t>(A->n_rows, 1), 256);
    ell_count_kernel<<<grid, 256, 0, st>>>(A->n_rows, e.n_pad, e.K, e.col, cnt, 0);
    GKO_TRY(counts_to_csr(A, cnt, &off, st));
    ell_gather_kernel<<<grid, 256, 0, st>>>(A->n_rows, e.n_pad, e.K, e.col, e.val, off, A->csr.col, A->csr.val);
    GKO_CUDA(cudaFreeAsync(cnt, st));
    GKO_CUDA(cudaFreeAsync(off, st));
    GKO_CUDA(cudaGetLastError());
    return finish_csr(A, st);
}

// --------------------------------------------------------- CSR <-> SELL-P

__global__ void sellp_len_kernel(int64_t n_rows, int64_t S, int64_t f, int64_t n_slices,
                                 const int32_t* __restrict__ row_ptr, int64_t* __restrict__ w)
{
    const int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (s >= n_slices) return;
    int64_t m = 0;
    const int64_t r1 = min((s + 1) * S, n_rows);
    for (int64_t r = s * S; r < r1; ++r) m = max(m, static_cast<int64_t>(row_ptr[r + 1] - row_ptr[r]));
    w[s] = (m + f - 1) / f * f;
}

__global__ void i64_to_i32_kernel(int64_t n, const int64_t* __restrict__ in, int32_t* __restrict__ out,
                                  uint32_t* err)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    if (in[i] > INT32_MAX) raise_error(err, kErrOverflow);
    out[i] = static_cast<int32_t>(in[i]);
}

// One thread per row slot of a slice (rows past n are all padding): slot k
// of row s*S + l at (slice_set[s] + k)*S + l gets the row's k-th entry or
// padding.  Consecutive threads write consecutive slots.
__global__ void csr_to_sellp_rows_kernel(int64_t n_rows, int64_t S, int64_t n_slices,
                                         const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                         const double* __restrict__ val, const int32_t* __restrict__ slen,
                                         const int32_t* __restrict__ sset, int32_t* __restrict__ scol,
                                         double* __restrict__ sval)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= n_slices * S) return;
    const int64_t s = r / S, l = r % S;
    const int64_t w = slen[s], base = static_cast<int64_t>(sset[s]) * S + l;
    int64_t a = 0, L = 0;
    if (r < n_rows) {
        a = row_ptr[r];
        L = row_ptr[r + 1] - a;
    }
    for (int64_t k = 0; k < w; ++k) {
        if (k < L) {
            scol[base + k * S] = col[a + k];
            sval[base + k * S] = val[a + k];
        } else {
            scol[base + k * S] = -1;
            sval[base + k * S] = 0.0;
        }
    }
}

int convert_csr_to_sellp(gko_matrix* A, cudaStream_t st)
{
    free_format(A, GKO_FMT_SELLP);
    SellpPart& s = A->sellp;
    s.S = A->sellp_S;
    s.f = A->sellp_f;
    s.n_slices = (A->n_rows + s.S - 1) / s.S;
    int64_t* w = nullptr;
    int64_t* off = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&w), (s.n_slices + 1) * sizeof(int64_t), st));
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&off), (s.n_slices + 1) * sizeof(int64_t), st));
    const int gs = ceil_div(std::max<int64_t>(s.n_slices, 1), 256);
    sellp_len_kernel<<<gs, 256, 0, st>>>(A->n_rows, s.S, s.f, s.n_slices, A->csr.row_ptr, w);
    GKO_TRY(exclusive_scan(w, off, s.n_slices, st));
    int64_t total_w = 0;
    GKO_TRY(read_back(&total_w, off + s.n_slices, st));
    if (total_w > INT32_MAX) {
        cudaFreeAsync(w, st);
        cudaFreeAsync(off, st);
        return fail(GKO_ERR_FORMAT_TOO_LARGE, "SELL-P slice offsets exceed int32");
    }
    s.slots = total_w * s.S;
    const double limit = std::max(A->ell_factor * static_cast<double>(A->nnz), static_cast<double>(1 << 22));
    if (static_cast<double>(s.slots) > limit) {
        cudaFreeAsync(w, st);
        cudaFreeAsync(off, st);
        s.slots = s.n_slices = 0;
        return fail(GKO_ERR_FORMAT_TOO_LARGE, "SELL-P padding exceeds the size limit (slots > max(factor * nnz, 2^22))");
    }
    GKO_TRY(dev_alloc(&s.slice_len, s.n_slices + 1));
    GKO_TRY(dev_alloc(&s.slice_set, s.n_slices + 1));
    i64_to_i32_kernel<<<gs, 256, 0, st>>>(s.n_slices, w, s.slice_len, A->d_err);
    i64_to_i32_kernel<<<ceil_div(s.n_slices + 1, 256), 256, 0, st>>>(s.n_slices + 1, off, s.slice_set, A->d_err);
    const int64_t alloc = padded_len(s.slots);
    GKO_TRY(dev_alloc(&s.col, alloc));
    GKO_TRY(dev_alloc(&s.val, alloc));
    GKO_CUDA(cudaMemsetAsync(s.col + s.slots, 0, (alloc - s.slots) * sizeof(int32_t), st));
    GKO_CUDA(cudaMemsetAsync(s.val + s.slots, 0, (alloc - s.slots) * sizeof(double), st));
    if (s.n_slices > 0)
        csr_to_sellp_rows_kernel<<<ceil_div(s.n_slices * s.S, 256), 256, 0, st>>>(
            A->n_rows, s.S, s.n_slices, A->csr.row_ptr, A->csr.col, A->csr.val, s.slice_len, s.slice_set, s.col,
            s.val);
    GKO_CUDA(cudaFreeAsync(w, st));
    GKO_CUDA(cudaFreeAsync(off, st));
    GKO_CUDA(cudaGetLastError());
    GKO_CUDA(cudaStreamSynchronize(st));
    A->has[GKO_FMT_SELLP] = true;
    return GKO_OK;
}

__global__ void sellp_count_kernel(int64_t n_rows, int64_t S, const int32_t* __restrict__ slen,
                                   const int32_t* __restrict__ sset, const int32_t* __restrict__ scol,
                                   int64_t* __restrict__ cnt)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= n_rows) return;
    const int64_t s = r / S, l = r % S, base = static_cast<int64_t>(sset[s]) * S + l;
    int64_t c = 0;
    for (int64_t k = 0; k < slen[s]; ++k) c += scol[base + k * S] >= 0;
    cnt[r] = c;
}

__global__ void sellp_gather_kernel(int64_t n_rows, int64_t S, const int32_t* __restrict__ slen,
                                    const int32_t* __restrict__ sset, const int32_t* __restrict__ scol,
                                    const double* __restrict__ sval, const int64_t* __restrict__ off,
                                    int32_t* __restrict__ col, double* __restrict__ val)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= n_rows) return;
    const int64_t s = r / S, l = r % S, base = static_cast<int64_t>(sset[s]) * S + l;
    int64_t o = off[r];
    for (int64_t k = 0; k < slen[s]; ++k) {
        const int32_t c = scol[base + k * S];
        if (c < 0) continue;
        col[o] = c;
        val[o] = sval[base + k * S];
        ++o;
    }
}

int convert_sellp_to_csr(gko_matrix* A, cudaStream_t st)
{
    free_format(A, GKO_FMT_CSR);
    const SellpPart& s = A->sellp;
    int64_t* cnt = nullptr;
    int64_t* off = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&cnt), (A->n_rows + 1) * sizeof(int64_t), st));
    const int grid = ceil_div(std::max<int64_t>(A->n_rows, 1), 256);
    sellp_count_kernel<<<grid, 256, 0, st>>>(A->n_rows, s.S, s.slice_len, s.slice_set, s.col, cnt);
    GKO_TRY(counts_to_csr(A, cnt, &off, st));
    sellp_gather_kernel<<<grid, 256, 0, st>>>(A->n_rows, s.S, s.slice_len, s.slice_set, s.col, s.val, off,
                                              A->csr.col, A->csr.val);
    GKO_CUDA(cudaFreeAsync(cnt, st));
    GKO_CUDA(cudaFreeAsync(off, st));
    GKO_CUDA(cudaGetLastError());
    return finish_csr(A, st);
}

// --------------------------------------------------------- CSR <-> hybrid

// Row-length histogram: shared-memory bins for lengths < 4096 (flushed
// once per block), global atomics for longer rows.  Integer counts: the
// result does not depend on the order of the additions.
constexpr int kHistShared = 4096;
__global__ void len_hist_kernel(int64_t n_rows, int64_t kmax, const int32_t* __restrict__ row_ptr,
                                int64_t* __restrict__ hist)
{
    __shared__ unsigned int sh[kHistShared];
    const int nb = static_cast<int>(min(kmax + 1, static_cast<int64_t>(kHistShared)));
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n_rows;
         r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int L = row_ptr[r + 1] - row_ptr[r];
        if (L < nb)
            atomicAdd(&sh[L], 1u);
        else
            atomicAdd(reinterpret_cast<unsigned long long*>(hist + L), 1ull);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (sh[i]) atomicAdd(reinterpret_cast<unsigned long long*>(hist + i), static_cast<unsigned long long>(sh[i]));
}

// K_h = argmin_K n_pad*K*(s_v+4) + overflow(K)*(s_v+8), ties to smaller K,
// with overflow(K) = sum_{L > K} (L - K) hist[L].  One block of 1024
// threads: thread t owns the lengths of a contiguous chunk, the counts of
// longer rows come from a suffix scan of the chunk totals, each thread
// walks its chunk downwards, and a block argmin picks the best K.  Byte
// counts are integers below 2^53, so the double arithmetic is exact and
// the choice is the same as any sequential evaluation.
constexpr int kWidthThreads = 1024;
__global__ void __launch_bounds__(kWidthThreads)
    hybrid_width_kernel(int64_t kmax, int64_t n_pad, int64_t s_v, const int64_t* __restrict__ hist,
                        int64_t* __restrict__ out)
{
    __shared__ int64_t s_cnt[kWidthThreads], s_sum[kWidthThreads];
    __shared__ double s_best[kWidthThreads];
    __shared__ int64_t s_bk[kWidthThreads];
    const int t = threadIdx.x;
    const int64_t nbins = kmax + 1;
    const int64_t ch = (nbins + kWidthThreads - 1) / kWidthThreads;
    const int64_t c0 = t * ch, c1 = min(c0 + ch, nbins);
    int64_t cnt = 0, sum = 0;
    for (int64_t L = c0; L < c1; ++L) {
        cnt += hist[L];
        sum += L * hist[L];
    }
    s_cnt[t] = cnt;
    s_sum[t] = sum;
    __syncthreads();
    // inclusive suffix scan over threads (Hillis-Steele on integers)
    for (int o = 1; o < kWidthThreads; o <<= 1) {
        const int64_t a = t + o < kWidthThreads ? s_cnt[t + o] : 0;
        const int64_t b = t + o < kWidthThreads ? s_sum[t + o] : 0;
        __syncthreads();
        s_cnt[t] += a;
        s_sum[t] += b;
        __syncthreads();
    }
    // rows with length >= c1 (chunks after this one)
    int64_t cnt_gt = t + 1 < kWidthThreads ? s_cnt[t + 1] : 0;
    int64_t sum_gt = t + 1 < kWidthThreads ? s_sum[t + 1] : 0;
    double best = -1.0;
    int64_t best_k = -1;
    for (int64_t K = c1 - 1; K >= c0; --K) {
        if (K + 1 < c1) {  // hist[K + 1] of this chunk joins the "longer than K" rows
            cnt_gt += hist[K + 1];
            sum_gt += (K + 1) * hist[K + 1];
        }
        const int64_t over = sum_gt - K * cnt_gt;
        const double bytes = static_cast<double>(n_pad) * static_cast<double>(K) * static_cast<double>(s_v + 4) +
                             static_cast<double>(over) * static_cast<double>(s_v + 8);
        if (best < 0.0 || bytes <= best) {
            best = bytes;
            best_k = K;
        }
    }
    s_best[t] = best;
    s_bk[t] = best_k;
    __syncthreads();
    for (int o = kWidthThreads / 2; o; o >>= 1) {
        if (t < o) {
            const double b2 = s_best[t + o];
            const int64_t k2 = s_bk[t + o];
            const bool take = k2 >= 0 && (s_bk[t] < 0 || b2 < s_best[t] || (b2 == s_best[t] && k2 < s_bk[t]));
            if (take) {
                s_best[t] = b2;
                s_bk[t] = k2;
            }
        }
        __syncthreads();
    }
    if (t == 0) out[0] = s_bk[0] < 0 ? 0 : s_bk[0];
}

__global__ void overflow_count_kernel(int64_t n_rows, int64_t K, const int32_t* __restrict__ row_ptr,
                                      int64_t* __restrict__ cnt)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= n_rows) return;
    cnt[r] = max(static_cast<int64_t>(0), static_cast<int64_t>(row_ptr[r + 1] - row_ptr[r]) - K);
}

__global__ void csr_to_hybrid_coo_kernel(int64_t nnz, int64_t n_rows, int64_t K, const int32_t* __restrict__ row_ptr,
                                         const int32_t* __restrict__ thr_row, const int32_t* __restrict__ col,
                                         const double* __restrict__ val, const int64_t* __restrict__ off,
                                         int32_t* __restrict__ crow, int32_t* __restrict__ ccol,
                                         double* __restrict__ cval)
{
    const int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    for_entries(g, kSegP, nnz, n_rows, row_ptr, thr_row, [&](int64_t k, int64_t r, int64_t j) {
        if (j >= K) {
            const int64_t o = off[r] + (j - K);
            crow[o] = static_cast<int32_t>(r);
            ccol[o] = col[k];
            cval[o] = val[k];
        }
    });
}

int convert_csr_to_hybrid(gko_matrix* A, cudaStream_t st)
{
    free_format(A, GKO_FMT_HYBRID);
    HybridPart& h = A->hyb;
    const int64_t kmax = A->csr.max_len;
    int64_t* hist = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&hist), (kmax + 2) * sizeof(int64_t), st));
    GKO_CUDA(cudaMemsetAsync(hist, 0, (kmax + 2) * sizeof(int64_t), st));
    const int grid = ceil_div(std::max<int64_t>(A->n_rows, 1), 256);
    if (A->n_rows > 0)
        len_hist_kernel<<<std::min(grid, 152 * 2), 256, 0, st>>>(A->n_rows, kmax, A->csr.row_ptr, hist);
    const int64_t n_pad = (A->n_rows + 31) / 32 * 32;
    hybrid_width_kernel<<<1, kWidthThreads, 0, st>>>(kmax, n_pad, 8, hist, hist + kmax + 1);
    int64_t K = 0;
    GKO_TRY(read_back(&K, hist + kmax + 1, st));
    GKO_CUDA(cudaFreeAsync(hist, st));
    GKO_TRY(ell_fill(A, &h.ell, K, st));
    // COO part: per-row overflow counts -> offsets
    int64_t* cnt = nullptr;
    int64_t* off = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&cnt), (A->n_rows + 1) * sizeof(int64_t), st));
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&off), (A->n_rows + 1) * sizeof(int64_t), st));
    if (A->n_rows > 0) overflow_count_kernel<<<grid, 256, 0, st>>>(A->n_rows, K, A->csr.row_ptr, cnt);
    GKO_TRY(exclusive_scan(cnt, off, A->n_rows, st));
    int64_t over = 0;
    GKO_TRY(read_back(&over, off + A->n_rows, st));
    CooPart& c = h.coo;
    c.nnz = over;
    const int64_t alloc = padded_len(over);
    GKO_TRY(dev_alloc(&c.row, alloc));
    GKO_TRY(dev_alloc(&c.col, alloc));
    GKO_TRY(dev_alloc(&c.val, alloc));
    GKO_CUDA(cudaMemsetAsync(c.row, 0, alloc * sizeof(int32_t), st));
    GKO_CUDA(cudaMemsetAsync(c.col, 0, alloc * sizeof(int32_t), st));
    GKO_CUDA(cudaMemsetAsync(c.val, 0, alloc * sizeof(double), st));
    const int64_t n_thr = (A->nnz + kSegP - 1) / kSegP;
    if (over > 0 && n_thr > 0)
        csr_to_hybrid_coo_kernel<<<ceil_div(n_thr, 256), 256, 0, st>>>(A->nnz, A->n_rows, K, A->csr.row_ptr,
                                                                        A->csr.thr_row, A->csr.col, A->csr.val, off,
                                                                        c.row, c.col, c.val);
    c.P = coo_entries_per_thread(A);
    GKO_TRY(seg_alloc(&c.seg, c.nnz, c.P, kSegThreadsCoo));
    GKO_CUDA(cudaFreeAsync(cnt, st));
    GKO_CUDA(cudaFreeAsync(off, st));
    GKO_CUDA(cudaGetLastError());
    GKO_CUDA(cudaStreamSynchronize(st));
    A->has[GKO_FMT_HYBRID] = true;
    return GKO_OK;
}

// per-row count of COO entries (rows sorted): upper_bound - lower_bound
__global__ void coo_count_kernel(int64_t n_rows, int64_t nnz, const int32_t* __restrict__ row,
                                 int64_t* __restrict__ cnt, int64_t* __restrict__ start)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= n_rows) return;
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (row[mid] < r) lo = mid + 1; else hi = mid;
    }
    const int64_t a = lo;
    hi = nnz;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (row[mid] <= r) lo = mid + 1; else hi = mid;
    }
    cnt[r] += lo - a;
    start[r] = a;
}

__global__ void hybrid_gather_kernel(int64_t n_rows, int64_t n_pad, int64_t K, const int32_t* __restrict__ ecol,
                                     const double* __restrict__ eval, const int32_t* __restrict__ ccol,
                                     const double* __restrict__ cval, const int64_t* __restrict__ cstart,
                                     const int64_t* __restrict__ off, int32_t* __restrict__ col,
                                     double* __restrict__ val)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= n_rows) return;
    int64_t o = off[r];
    for (int64_t k = 0; k < K; ++k) {
        const int32_t c = ecol[k * n_pad + r];
        if (c < 0) continue;
        col[o] = c;
        val[o] = eval[k * n_pad + r];
        ++o;
    }
    for (int64_t q = cstart[r]; o < off[r + 1]; ++q, ++o) {
        col[o] = ccol[q];
        val[o] = cval[q];
    }
}

int convert_hybrid_to_csr(gko_matrix* A, cudaStream_t st)
{
    free_format(A, GKO_FMT_CSR);
    const HybridPart& h = A->hyb;
    int64_t* cnt = nullptr;
    int64_t* cstart = nullptr;
    int64_t* off = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&cnt), (A->n_rows + 1) * sizeof(int64_t), st));
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&cstart), (A->n_rows + 1) * sizeof(int64_t), st));
    const int grid = ceil_div(std::max<int64_t>(A->n_rows, 1), 256);
    ell_count_kernel<<<grid, 256, 0, st>>>(A->n_rows, h.ell.n_pad, h.ell.K, h.ell.col, cnt, 0);
    coo_count_kernel<<<grid, 256, 0, st>>>(A->n_rows, h.coo.nnz, h.coo.row, cnt, cstart);
    GKO_TRY(counts_to_csr(A, cnt, &off, st));
    hybrid_gather_kernel<<<grid, 256, 0, st>>>(A->n_rows, h.ell.n_pad, h.ell.K, h.ell.col, h.ell.val, h.coo.col,
                                               h.coo.val, cstart, off, A->csr.col, A->csr.val);
    GKO_CUDA(cudaFreeAsync(cnt, st));
    GKO_CUDA(cudaFreeAsync(cstart, st));
    GKO_CUDA(cudaFreeAsync(off, st));
    GKO_CUDA(cudaGetLastError());
    return finish_csr(A, st);
}

// ------------------------------------------------------------ validation

// Flags: bit 0 row_ptr[0] != 0 or row_ptr[n] != nnz; bit 1 row_ptr not
// monotone; bit 2 column out of range; bit 3 columns not strictly ascending.
__global__ void validate_rows_kernel(int64_t n_rows, int64_t nnz, const int32_t* __restrict__ row_ptr,
                                     uint32_t* __restrict__ flags)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r == 0 && (row_ptr[0] != 0 || row_ptr[n_rows] != nnz)) atomicOr(flags, 1u);
    if (r >= n_rows) return;
    const int32_t a = row_ptr[r], b = row_ptr[r + 1];
    if (b < a || a < 0 || b > nnz) atomicOr(flags, 2u);
}

// entry-parallel (equal chunks of entries, any row lengths): columns in
// range and strictly ascending within each row
__global__ void validate_entries_kernel(int64_t n_rows, int64_t n_cols, int64_t nnz,
                                        const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ thr_row,
                                        const int32_t* __restrict__ col, uint32_t* __restrict__ flags)
{
    const int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    uint32_t f = 0;
    for_entries(g, kSegP, nnz, n_rows, row_ptr, thr_row, [&](int64_t k, int64_t, int64_t j) {
        const int32_t c = col[k];
        if (c < 0 || c >= n_cols) f |= 4u;
        if (j > 0 && c <= col[k - 1]) f |= 8u;
    });
    if (f) atomicOr(flags, f);
}

int compute_thr_row(int64_t n_rows, int64_t nnz, const int32_t* row_ptr, int32_t* thr_row, cudaStream_t st);

int validate_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                 cudaStream_t st)
{
    uint32_t* d = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(uint32_t), st));
    GKO_CUDA(cudaMemsetAsync(d, 0, sizeof(uint32_t), st));
    validate_rows_kernel<<<ceil_div(std::max<int64_t>(n_rows, 1), 256), 256, 0, st>>>(n_rows, nnz, row_ptr, d);
    uint32_t h = 0;
    GKO_TRY(read_back(&h, d, st));
    if (h == 0 && nnz > 0) {  // row pointers are valid: split the entries evenly
        const int64_t n_thr = (nnz + kSegP - 1) / kSegP;
        int32_t* tr = nullptr;
        GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&tr), n_thr * sizeof(int32_t), st));
        GKO_TRY(compute_thr_row(n_rows, nnz, row_ptr, tr, st));
        validate_entries_kernel<<<ceil_div(n_thr, 256), 256, 0, st>>>(n_rows, n_cols, nnz, row_ptr, tr, col, d);
        GKO_TRY(read_back(&h, d, st));
        GKO_CUDA(cudaFreeAsync(tr, st));
    }
    GKO_CUDA(cudaFreeAsync(d, st));
    GKO_CUDA(cudaGetLastError());
    if (h) {
        const char* why = (h & 1)   ? "row_ptr[0] != 0 or row_ptr[n] != nnz"
                          : (h & 2) ? "row_ptr is not monotone"
                          : (h & 4) ? "column index out of range"
                                    : "column indices not strictly ascending within a row";
        return fail(GKO_ERR_INVALID_MATRIX, why);
    }
    return GKO_OK;
}

// ------------------------------------------------------------- freeing

void free_format(gko_matrix* A, int fmt)
{
    switch (fmt) {
        case GKO_FMT_CSR:
            dev_free(A->csr.row_ptr);
            dev_free(A->csr.col);
            dev_free(A->csr.val);
            dev_free(A->csr.thr_row);
            dev_free(A->csr.bin_rows);
            dev_free(A->csr.bin_tasks);
            A->csr.n_bin_tasks = 0;
            seg_free(&A->csr.seg);
            break;
        case GKO_FMT_COO:
            dev_free(A->coo.row);
            dev_free(A->coo.col);
            dev_free(A->coo.val);
            seg_free(&A->coo.seg);
            A->coo.nnz = 0;
            break;
        case GKO_FMT_ELL:
            dev_free(A->ell.col);
            dev_free(A->ell.val);
            A->ell.K = A->ell.n_pad = 0;
            break;
        case GKO_FMT_SELLP:
            dev_free(A->sellp.slice_len);
            dev_free(A->sellp.slice_set);
            dev_free(A->sellp.col);
            dev_free(A->sellp.val);
            A->sellp.slots = A->sellp.n_slices = 0;
            break;
        case GKO_FMT_HYBRID:
            dev_free(A->hyb.ell.col);
            dev_free(A->hyb.ell.val);
            dev_free(A->hyb.coo.row);
            dev_free(A->hyb.coo.col);
            dev_free(A->hyb.coo.val);
            seg_free(&A->hyb.coo.seg);
            A->hyb.coo.nnz = 0;
            A->hyb.ell.K = 0;
            break;
        default: break;
    }
    if (fmt >= 0 && fmt < 5) A->has[fmt] = false;
}

}  // namespace gko
