// Block-Jacobi preconditioner for the Krylov solvers of the paper's Sec. 6.2
// (the paper benchmarks the solvers without defining a preconditioner; this
// is the textbook block-Jacobi of Saad, Iterative Methods for Sparse Linear
// Systems, Sec. 10.2): M = blockdiag(A_11, ..., A_kk), the diagonal blocks
// of A on runs of consecutive rows, inverted once, applied as z = M^-1 r.
//
// Generation:
//   * supervariables: a flag per row, set when its stored column list
//     differs from the previous row's (one thread per row);
//   * blocks: the runs are cut at max_bs rows and merged greedily in row
//     order while a block stays at most max_bs rows -- a sequential scan of
//     the flags on the host (n bytes copied back once);
//   * inverses: one warp per block, lane i owning row i of [B | I] in
//     shared memory, Gauss-Jordan elimination with partial pivoting (the
//     pivot row found by a warp arg-max), FP64.  Entry (i, j) of the inverse
//     of the block starting at row o with s rows goes to
//     inv[o * max_bs + j * s + i]: a block's s * s entries are contiguous
//     and column-major, so the threads of its rows read one column at a time
//     with consecutive addresses.
// Application: one thread per row, z_i = sum_j inv(i, j) r_(o+j); threads
// of one block read the same r entries (L1 broadcast).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "solver.cuh"

namespace gko {

constexpr int kBjWarps = 4;  // warps (blocks inverted at once) per CTA

// flag[i] = 1 when row i starts a run of identical column lists
__global__ void bj_flags_kernel(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                uint8_t* __restrict__ flag)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint8_t f = 1;
        if (i > 0) {
            const int32_t a = row_ptr[i - 1], b = row_ptr[i], e = row_ptr[i + 1];
            if (b - a == e - b) {
                f = 0;
                for (int32_t k = 0; k < e - b; ++k)
                    if (col[a + k] != col[b + k]) {
                        f = 1;
                        break;
                    }
            }
        }
        flag[i] = f;
    }
}

// row_block[r] = k for the rows of block k (thread per block)
__global__ void bj_row_block_kernel(int64_t n_blocks, const int32_t* __restrict__ bp, int32_t* __restrict__ row_block)
{
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n_blocks;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x)
        for (int32_t r = bp[k]; r < bp[k + 1]; ++r) row_block[r] = static_cast<int32_t>(k);
}

// One warp per diagonal block.  Shared memory per warp: B and E, s x s
// each, row stride bs + 1.  A zero (or NaN) pivot sets *singular and leaves
// that block's inverse unwritten.
__global__ void __launch_bounds__(kBjWarps * 32)
    bj_invert_kernel(int64_t n_blocks, const int32_t* __restrict__ bp, const int32_t* __restrict__ row_ptr,
                     const int32_t* __restrict__ col, const double* __restrict__ val, int bs,
                     double* __restrict__ inv, int32_t* singular)
{
    extern __shared__ double bj_smem[];
    const int w = static_cast<int>(threadIdx.x / 32), lane = static_cast<int>(threadIdx.x % 32);
    const int ld = bs + 1;
    double* B = bj_smem + static_cast<int64_t>(w) * 2 * bs * ld;
    double* E = B + bs * ld;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * kBjWarps + w; k < n_blocks;
         k += static_cast<int64_t>(gridDim.x) * kBjWarps) {  // warp-uniform
        const int64_t o = bp[k];
        const int s = bp[k + 1] - static_cast<int32_t>(o);
        if (lane < s) {
            double* Bi = B + lane * ld;
            double* Ei = E + lane * ld;
            for (int j = 0; j < s; ++j) {
                Bi[j] = 0.0;
                Ei[j] = j == lane ? 1.0 : 0.0;
            }
            for (int32_t e = row_ptr[o + lane]; e < row_ptr[o + lane + 1]; ++e) {
                const int64_t c = static_cast<int64_t>(col[e]) - o;
                if (c >= 0 && c < s) Bi[c] += val[e];  // duplicates summed, as the products do
            }
        }
        __syncwarp();
        bool ok = true;
        for (int c = 0; c < s; ++c) {
            // pivot row: largest |B(i, c)| over c <= i < s, lowest i on ties
            double mag = (lane >= c && lane < s) ? fabs(B[lane * ld + c]) : -1.0;
            int arg = lane;
            for (int off = 16; off; off >>= 1) {
                const double om = __shfl_xor_sync(0xffffffffu, mag, off);
                const int oa = __shfl_xor_sync(0xffffffffu, arg, off);
                if (om > mag || (om == mag && oa < arg)) {
                    mag = om;
                    arg = oa;
                }
            }
            if (!(mag > 0.0)) {  // the same on every lane
                ok = false;
                break;
            }
            if (arg != c && lane < s) {  // lane j swaps column j of rows c and arg
                double t = B[c * ld + lane];
                B[c * ld + lane] = B[arg * ld + lane];
                B[arg * ld + lane] = t;
                t = E[c * ld + lane];
                E[c * ld + lane] = E[arg * ld + lane];
                E[arg * ld + lane] = t;
            }
            __syncwarp();
            const double piv = B[c * ld + c];
            __syncwarp();
            if (lane < s) {
                B[c * ld + lane] /= piv;
                E[c * ld + lane] /= piv;
            }
            __syncwarp();
            if (lane < s && lane != c) {
                double* Bi = B + lane * ld;
                double* Ei = E + lane * ld;
                const double f = Bi[c];
                for (int j = 0; j < s; ++j) {
                    Bi[j] = fma(-f, B[c * ld + j], Bi[j]);
                    Ei[j] = fma(-f, E[c * ld + j], Ei[j]);
                }
            }
            __syncwarp();
        }
        if (!ok) {
            if (lane == 0) atomicOr(singular, 1);
            __syncwarp();
            continue;
        }
        if (lane < s) {
            double* dst = inv + o * bs + lane;
            for (int j = 0; j < s; ++j) dst[static_cast<int64_t>(j) * s] = E[lane * ld + j];
        }
        __syncwarp();
    }
}

__device__ __forceinline__ double bj_row(int64_t i, const int32_t* __restrict__ row_block,
                                         const int32_t* __restrict__ bp, const double* __restrict__ inv, int bs,
                                         const double* __restrict__ r)
{
    const int32_t k = row_block[i];
    const int64_t o = bp[k];
    const int s = bp[k + 1] - static_cast<int32_t>(o);
    const double* m = inv + o * bs + (i - o);
    double acc = 0.0;
    for (int j = 0; j < s; ++j) acc = fma(__ldg(m + static_cast<int64_t>(j) * s), __ldg(r + o + j), acc);
    return acc;
}

__global__ void bj_apply_kernel(int64_t n, const int32_t* __restrict__ row_block, const int32_t* __restrict__ bp,
                                const double* __restrict__ inv, int bs, const double* __restrict__ r,
                                double* __restrict__ z)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        z[i] = bj_row(i, row_block, bp, inv, bs, r);
}

// z = M^-1 r with rho' = r.z (and ||r||^2) in one grid reduction
__global__ void __launch_bounds__(kRedThreads)
    bj_z_kernel(int64_t n, const int32_t* __restrict__ row_block, const int32_t* __restrict__ bp,
                const double* __restrict__ inv, int bs, const double* __restrict__ r, double* __restrict__ z,
                SolverState* s, double* part, cudaGraphConditionalHandle h, int mode, int force)
{
    if (s->done && !force) return;  // set only by the last block of an earlier kernel
    double rz = 0.0, rr = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kRedThreads) {
        const double zi = bj_row(i, row_block, bp, inv, bs, r);
        z[i] = zi;
        const double ri = r[i];
        rz = fma(ri, zi, rz);
        rr = fma(ri, ri, rr);
    }
    grid_sum2(rz, rr, part, &s->ticket, [&](double rz_t, double rr_t) {
        if (mode == kBjInit) {
            s->rho = rz_t;
            s->rho0 = rz_t;
            s->dot_out = rr_t;
            if (sqrt(rr_t) <= s->tol * s->stop_ref) {
                s->conv = 1;
                s->status = GKO_OK;
                s->done = 1;
            }
            return;
        }
        if (!(rz_t == rz_t)) {
            s->status = GKO_ERR_BREAKDOWN;
            stop_loop(s, h);
            return;
        }
        s->beta = rz_t / s->rho;
        s->rho = rz_t;
    });
}

void bj_z_launch(const gko_block_jacobi* M, const double* r, double* z, SolverState* s, double* part, int grid,
                 cudaGraphConditionalHandle h, int mode, int force, cudaStream_t st)
{
    bj_z_kernel<<<grid, kRedThreads, 0, st>>>(M->n_rows, M->row_block, M->block_ptr, M->inv, M->max_bs, r, z, s,
                                              part, h, mode, force);
}

static int elem_grid(int64_t n, int threads)
{
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads,
                                                                    static_cast<int64_t>(device_sm_count()) * 16)));
}

}  // namespace gko

using namespace gko;

extern "C" int gko_block_jacobi_destroy(gko_block_jacobi* M)
{
    if (!M) return GKO_OK;
    dev_free(M->block_ptr);
    dev_free(M->row_block);
    dev_free(M->inv);
    delete M;
    return GKO_OK;
}

extern "C" int gko_block_jacobi_create(const gko_matrix* A, int max_block_size, void* stream, gko_block_jacobi** out)
{
    if (!A || !out) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (max_block_size < 1 || max_block_size > 32) return fail(GKO_ERR_INVALID_ARG, "max_block_size must be in 1..32");
    if (A->n_rows != A->n_cols) return fail(GKO_ERR_DIM_MISMATCH, "block-Jacobi needs a square matrix");
    if (!A->has[GKO_FMT_CSR]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "the preconditioner reads the CSR part");
    int dev = -1;
    GKO_CUDA(cudaGetDevice(&dev));
    if (dev != A->device) return fail(GKO_ERR_INVALID_ARG, "handle used on another device than it was created on");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = A->n_rows;
    const int bs = max_block_size;
    gko_block_jacobi* M = new gko_block_jacobi();
    M->device = dev;
    M->n_rows = n;
    M->max_bs = bs;
    uint8_t* flag = nullptr;
    int32_t* singular = nullptr;
    auto cleanup = [&](int s) {
        dev_free(flag);
        dev_free(singular);
        gko_block_jacobi_destroy(M);
        return s;
    };
    int s;
    // supervariable starts, then the greedy merge on the host
    std::vector<int32_t> bp(1, 0);
    if (n > 0) {
        if ((s = dev_alloc(&flag, n)) != GKO_OK) return cleanup(s);
        bj_flags_kernel<<<elem_grid(n, 256), 256, 0, st>>>(n, A->csr.row_ptr, A->csr.col, flag);
        std::vector<uint8_t> hf(n);
        cudaError_t e = cudaMemcpyAsync(hf.data(), flag, n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "block-Jacobi supervariables"));
        int64_t blk = 0, piece = 0;  // starts of the current block and of the current piece
        for (int64_t i = 1; i <= n; ++i) {
            if (i < n && !hf[i] && i - piece < bs) continue;
            // the piece [piece, i) is complete: it joins the block or opens one
            if (i - blk > bs) {
                bp.push_back(static_cast<int32_t>(piece));
                blk = piece;
            }
            piece = i;
        }
        bp.push_back(static_cast<int32_t>(n));
    }
    M->n_blocks = static_cast<int64_t>(bp.size()) - 1;
    if ((s = dev_alloc(&M->block_ptr, M->n_blocks + 1)) != GKO_OK || (s = dev_alloc(&M->row_block, n)) != GKO_OK ||
        (s = dev_alloc(&M->inv, n * bs)) != GKO_OK || (s = dev_alloc(&singular, 1)) != GKO_OK)
        return cleanup(s);
    cudaError_t e = cudaMemcpyAsync(M->block_ptr, bp.data(), bp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->inv, 0, static_cast<size_t>(std::max<int64_t>(n, 1)) * bs * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(singular, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "block-Jacobi set-up"));
    int32_t hsing = 0;
    if (M->n_blocks > 0) {
        bj_row_block_kernel<<<elem_grid(M->n_blocks, 256), 256, 0, st>>>(M->n_blocks, M->block_ptr, M->row_block);
        const int smem = kBjWarps * 2 * bs * (bs + 1) * static_cast<int>(sizeof(double));
        e = smem_limit_once(reinterpret_cast<const void*>(bj_invert_kernel), smem);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "block-Jacobi inversion shared memory"));
        const int grid = static_cast<int>(std::max<int64_t>(
            1, std::min<int64_t>((M->n_blocks + kBjWarps - 1) / kBjWarps, static_cast<int64_t>(device_sm_count()) * 16)));
        bj_invert_kernel<<<grid, kBjWarps * 32, smem, st>>>(M->n_blocks, M->block_ptr, A->csr.row_ptr, A->csr.col,
                                                            A->csr.val, bs, M->inv, singular);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hsing, singular, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "block-Jacobi generation"));
    if (hsing) return cleanup(fail(GKO_ERR_BREAKDOWN, "block-Jacobi: a diagonal block is singular (zero pivot)"));
    dev_free(flag);
    dev_free(singular);
    *out = M;
    return GKO_OK;
}

extern "C" int gko_block_jacobi_export(const gko_block_jacobi* M, int64_t* n_blocks, int32_t* block_ptr, double* inv,
                                       void* stream)
{
    if (!M || !n_blocks) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *n_blocks = M->n_blocks;
    if (block_ptr)
        GKO_CUDA(cudaMemcpyAsync(block_ptr, M->block_ptr, (M->n_blocks + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (inv && M->n_rows > 0)
        GKO_CUDA(cudaMemcpyAsync(inv, M->inv, M->n_rows * M->max_bs * sizeof(double), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    return GKO_OK;
}

extern "C" int gko_block_jacobi_apply(const gko_block_jacobi* M, const double* r, double* z, void* stream)
{
    if (!M) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (M->n_rows == 0) return GKO_OK;
    if (!r || !z) return fail(GKO_ERR_INVALID_ARG, "NULL vector");
    if (r == z) return fail(GKO_ERR_INVALID_ARG, "r and z must not overlap");
    int dev = -1;
    GKO_CUDA(cudaGetDevice(&dev));
    if (dev != M->device) return fail(GKO_ERR_INVALID_ARG, "preconditioner used on another device than it was created on");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bj_apply_kernel<<<elem_grid(M->n_rows, 256), 256, 0, st>>>(M->n_rows, M->row_block, M->block_ptr, M->inv,
                                                               M->max_bs, r, z);
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

extern "C" int gko_pcg_block_jacobi(const gko_matrix* A, int fmt, const gko_block_jacobi* M, const double* b,
                                    double* x, double tol, int maxit, void* stream, gko_solve_info* info)
{
    if (!A || !M) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (A->n_rows != A->n_cols) return fail(GKO_ERR_DIM_MISMATCH, "CG needs a square matrix");
    if (M->n_rows != A->n_rows) return fail(GKO_ERR_DIM_MISMATCH, "preconditioner built for another size");
    if (fmt < 0 || fmt > GKO_FMT_HYBRID) return fail(GKO_ERR_INVALID_ARG, "unknown format");
    if (!A->has[fmt]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "format not materialised");
    if (A->n_rows > 0 && (!b || !x)) return fail(GKO_ERR_INVALID_ARG, "NULL vector");
    if (!(tol >= 0.0) || maxit < 0) return fail(GKO_ERR_INVALID_ARG, "tol must be >= 0 and maxit >= 0");
    int dev = -1;
    GKO_CUDA(cudaGetDevice(&dev));
    if (dev != A->device || dev != M->device)
        return fail(GKO_ERR_INVALID_ARG, "handle used on another device than it was created on");
    return pcg_block_jacobi_solve(A, fmt, M, b, x, tol, maxit, static_cast<cudaStream_t>(stream), info);
}
