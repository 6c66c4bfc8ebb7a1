// Conjugate gradients for several right-hand sides at once, A X = B with
// X, B of k columns: k independent Hestenes-Stiefel recurrences (the CG of
// the paper's Sec. 6.2, one per column, each with its own alpha, beta and
// stop test) that share one sparse product per step, the multi-vector
// product (SpMM) of Sec. 6.1 applied to the k search directions.  Sharing
// the product reads the matrix once for the k columns; on GB300 the
// product is bound by the FP64 pipe (one FMA per entry and column), so the
// saving is the matrix and index traffic and the launches of k-1 products.
//
// Blocks are row-major (element (i, c) at i * ld + c); the workspace blocks
// R, P, Q have ld = k.  For k dividing 32 the vector kernels take a thread
// per element (coalesced; a thread always meets the same column); for other
// k a thread per row walks the row's k columns.  One step is six launches
// inside a CUDA-graph WHILE loop:
//   Q = A P                                       (SpMM)
//   per-column partial sums of P.Q                (thread per row, k columns)
//   alpha_c = rho_c / (P.Q)_c                     (one block, a warp per column)
//   X += alpha P, R -= alpha Q, partial |R_c|^2   (active columns only)
//   beta_c, rho_c, stop tests, loop condition     (one block)
//   P = R + beta P                                (active columns only)
// A column stops on its recursive residual |r_c| <= tol |b_c|; the host then
// confirms it with the FP64 true residual (up to four times, as gko_cg) and
// lets an unconfirmed column go on.  Per-column sums are formed in a fixed
// order (rows by thread, a reduce-scatter over the warp, warps, then blocks
// in index order), so results do not depend on scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "solver.cuh"

namespace gko {

constexpr int kMcMaxK = 32;       // columns per solve
constexpr int kMcThreads = 256;   // threads of the row kernels
constexpr int kMcFinal = 1024;    // threads of the finalising block (a warp per column)

enum { kMcIterating = 0, kMcConverged = 1, kMcDone = 2 };

struct MultiState {
    double rho[kMcMaxK], alpha[kMcMaxK], beta[kMcMaxK], stop_ref[kMcMaxK], val[kMcMaxK];
    int32_t phase[kMcMaxK];   // kMcIterating, kMcConverged (recursive residual met), kMcDone
    int32_t iters[kMcMaxK];   // steps taken by the column
    int32_t status[kMcMaxK];  // GKO_OK, GKO_ERR_NOT_CONVERGED or GKO_ERR_BREAKDOWN once done
    int32_t k, maxit;
    double tol;
};

// Warp sums of KM per-column accumulators (KM a power of two <= 32) by
// reduce-scatter: at distance D = 16, 8, ... each lane keeps the half of
// its columns picked by bit D of the lane (the upper half when it is set)
// and adds the partner's partials of them, then plain butterfly steps finish
// the sums: KM - 1 + 5 - log2(KM) FP64 adds per lane, where a butterfly per
// column would take 5 KM.  The steps are unrolled at compile time, so the
// accumulators stay in registers.
template <int K, int D>
struct McScatter {
    template <int KM>
    __device__ __forceinline__ static void run(double (&v)[KM], int lane, int& col)
    {
        const bool upper = (lane & D) != 0;
#pragma unroll
        for (int q = 0; q < K / 2; ++q) {
            const double send = upper ? v[q] : v[q + K / 2];
            const double keep = upper ? v[q + K / 2] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, D);
        }
        if (upper) col += K / 2;
        McScatter<K / 2, D / 2>::run(v, lane, col);
    }
};
template <int D>
struct McScatter<1, D> {
    template <int KM>
    __device__ __forceinline__ static void run(double (&v)[KM], int, int&)
    {
#pragma unroll
        for (int d = D; d; d >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], d);
    }
};

// part[blockIdx.x * kMcMaxK + c] = the block's sum of acc[c] over its
// threads, c < KM
template <int KM>
__device__ __forceinline__ void mc_block_partials(double (&acc)[KM], double* __restrict__ part)
{
    __shared__ double sh[KM][kMcThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int col = 0;
    McScatter<KM, 16>::run(acc, lane, col);
    // after log2(KM) scatter steps the lanes agreeing in the bits below them
    // hold the same column's sum: the lowest of them stores it
    constexpr int kLow = KM >= 32 ? 1 : 32 / KM;
    if ((lane & (kLow - 1)) == 0) sh[col][w] = acc[0];
    __syncthreads();
    if (threadIdx.x < KM) {
        double t = 0.0;
        for (int q = 0; q < kMcThreads / 32; ++q) t += sh[threadIdx.x][q];
        part[blockIdx.x * static_cast<int64_t>(kMcMaxK) + threadIdx.x] = t;
    }
}

// Sum of column c of the partials over nblocks blocks, by the warp that
// calls it (lanes stride over the blocks; then a butterfly); every lane
// returns the total.
__device__ __forceinline__ double mc_column_total(const double* __restrict__ part, int nblocks, int c)
{
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    for (int b = lane; b < nblocks; b += 32) t += __ldcg(part + b * static_cast<int64_t>(kMcMaxK) + c);
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// ------------------------------------------------------------- kernels

// per-column partial sums of P .* Q (rows by thread).  With k == KM the
// column loop has no bound test, so the compiler issues a row's loads
// together; otherwise each column is guarded.
template <int KM>
__global__ void __launch_bounds__(kMcThreads)
    mc_pq_partial_kernel(int64_t n, int k, const double* __restrict__ P, const double* __restrict__ Q,
                         double* __restrict__ part)
{
    double acc[KM];
#pragma unroll
    for (int c = 0; c < KM; ++c) acc[c] = 0.0;
    const bool full = k == KM;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kMcThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kMcThreads) {
        const double* p = P + i * k;
        const double* q = Q + i * k;
        if (full) {
#pragma unroll
            for (int c = 0; c < KM; ++c) acc[c] = fma(p[c], q[c], acc[c]);
        } else {
#pragma unroll
            for (int c = 0; c < KM; ++c)
                if (c < k) acc[c] = fma(p[c], q[c], acc[c]);
        }
    }
    mc_block_partials(acc, part);
}

// ------------------------------------- element kernels (k divides 32)
//
// Thread per element of the row-major block (consecutive threads,
// consecutive addresses), four elements per pass.  The grid's thread count
// is a multiple of 32, so a thread always meets the same column
// c = lane mod k and keeps one accumulator; lanes of equal c combine by a
// butterfly over the distances 16 .. k.

// the block's sums of a per-thread value by column (lane mod k) into
// part[blockIdx.x * kMcMaxK + c], c < k
__device__ __forceinline__ void mc_elem_partials(double acc, int k, double* __restrict__ part)
{
    __shared__ double sh[kMcMaxK][kMcThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = 16; d >= k; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if (lane < k) sh[lane][w] = acc;
    __syncthreads();
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int q = 0; q < kMcThreads / 32; ++q) t += sh[threadIdx.x][q];
        part[blockIdx.x * static_cast<int64_t>(kMcMaxK) + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kMcThreads)
    mc_pq_elem_kernel(int64_t ne, int k, const double* __restrict__ P, const double* __restrict__ Q,
                      double* __restrict__ part)
{
    const int64_t nth = static_cast<int64_t>(gridDim.x) * kMcThreads;
    int64_t e = blockIdx.x * static_cast<int64_t>(kMcThreads) + threadIdx.x;
    double acc = 0.0;
    for (; e + 3 * nth < ne; e += 4 * nth) {
        const double p0 = P[e], p1 = P[e + nth], p2 = P[e + 2 * nth], p3 = P[e + 3 * nth];
        const double q0 = Q[e], q1 = Q[e + nth], q2 = Q[e + 2 * nth], q3 = Q[e + 3 * nth];
        acc = fma(p3, q3, fma(p2, q2, fma(p1, q1, fma(p0, q0, acc))));
    }
    for (; e < ne; e += nth) acc = fma(P[e], Q[e], acc);
    mc_elem_partials(acc, k, part);
}

// X += alpha P, R -= alpha Q (iterating columns), partial sums of R .* R;
// X has leading dimension ldx
__global__ void __launch_bounds__(kMcThreads)
    mc_update_elem_kernel(int64_t ne, int k, double* __restrict__ X, int64_t ldx, double* __restrict__ R,
                          const double* __restrict__ P, const double* __restrict__ Q, const MultiState* s,
                          double* __restrict__ part)
{
    const int c = threadIdx.x % k;  // the thread's column (nth is a multiple of k)
    const bool on = s->phase[c] == kMcIterating;
    const double a = on ? s->alpha[c] : 0.0;
    const int64_t nth = static_cast<int64_t>(gridDim.x) * kMcThreads;
    int64_t e = blockIdx.x * static_cast<int64_t>(kMcThreads) + threadIdx.x;
    double acc = 0.0;
    const int lk = __ffs(k) - 1;  // k is a power of two
    auto xi = [&](int64_t el) { return (el >> lk) * ldx + c; };
    for (; e + 3 * nth < ne; e += 4 * nth) {
        double xv[4], rv[4], pv[4], qv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t el = e + u * nth;
            xv[u] = X[xi(el)];
            rv[u] = R[el];
            pv[u] = P[el];
            qv[u] = Q[el];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t el = e + u * nth;
            const double rn = on ? fma(-a, qv[u], rv[u]) : rv[u];
            X[xi(el)] = on ? fma(a, pv[u], xv[u]) : xv[u];
            R[el] = rn;
            acc = fma(rn, rn, acc);
        }
    }
    for (; e < ne; e += nth) {
        const double rn = on ? fma(-a, Q[e], R[e]) : R[e];
        if (on) X[xi(e)] = fma(a, P[e], X[xi(e)]);
        R[e] = rn;
        acc = fma(rn, rn, acc);
    }
    mc_elem_partials(acc, k, part);
}

// P = R + beta P (iterating columns; initial: P = R)
__global__ void __launch_bounds__(kMcThreads)
    mc_pupdate_elem_kernel(int64_t ne, int k, double* __restrict__ P, const double* __restrict__ R,
                           const MultiState* s, int initial)
{
    const int c = threadIdx.x % k;
    const bool on = initial || s->phase[c] == kMcIterating;
    const double b = initial ? 0.0 : s->beta[c];
    if (!on) return;  // nothing of this thread's column changes
    const int64_t nth = static_cast<int64_t>(gridDim.x) * kMcThreads;
    int64_t e = blockIdx.x * static_cast<int64_t>(kMcThreads) + threadIdx.x;
    for (; e + 3 * nth < ne; e += 4 * nth) {
        double pv[4], rv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            pv[u] = P[e + u * nth];
            rv[u] = R[e + u * nth];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) P[e + u * nth] = fma(b, pv[u], rv[u]);
    }
    for (; e < ne; e += nth) P[e] = fma(b, P[e], R[e]);
}

// alpha_c = rho_c / (P.Q)_c for the iterating columns; a non-positive or
// NaN P.Q ends the column with a breakdown
__global__ void __launch_bounds__(kMcFinal)
    mc_alpha_kernel(int nblocks, const double* __restrict__ part, MultiState* s)
{
    const int c = threadIdx.x >> 5;
    if (c >= s->k) return;  // warp-uniform
    const double pq = mc_column_total(part, nblocks, c);
    if ((threadIdx.x & 31) != 0 || s->phase[c] != kMcIterating) return;
    s->iters[c] += 1;
    if (!(pq > 0.0)) {
        s->alpha[c] = 0.0;
        s->phase[c] = kMcDone;
        s->status[c] = GKO_ERR_BREAKDOWN;
    } else {
        s->alpha[c] = s->rho[c] / pq;
    }
}

// X += alpha P, R -= alpha Q for the iterating columns; per-column partial
// sums of R .* R.  With k == KM every value of a row is loaded before any
// store (so the loads issue together) and a stopped column keeps its
// values by a select; with k < KM each column is guarded.
template <int KM>
__global__ void __launch_bounds__(kMcThreads)
    mc_update_kernel(int64_t n, int k, double* __restrict__ X, int64_t ldx, double* __restrict__ R,
                     const double* __restrict__ P, const double* __restrict__ Q, const MultiState* s,
                     double* __restrict__ part)
{
    __shared__ double al_s[kMcMaxK];
    __shared__ int on_s[kMcMaxK];
    if (threadIdx.x < kMcMaxK) {
        const bool it = threadIdx.x < k && s->phase[threadIdx.x] == kMcIterating;
        on_s[threadIdx.x] = it;
        al_s[threadIdx.x] = it ? s->alpha[threadIdx.x] : 0.0;
    }
    __syncthreads();
    double al[KM];
    bool on[KM];
#pragma unroll
    for (int c = 0; c < KM; ++c) {
        al[c] = al_s[c];
        on[c] = on_s[c] != 0;
    }
    double acc[KM];
#pragma unroll
    for (int c = 0; c < KM; ++c) acc[c] = 0.0;
    const bool full = k == KM;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kMcThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kMcThreads) {
        double* x = X + i * ldx;
        double* r = R + i * k;
        const double* p = P + i * k;
        const double* q = Q + i * k;
        if (full) {  // every load of the row first, then the stores
            double xv[KM], rv[KM], pv[KM], qv[KM];
#pragma unroll
            for (int c = 0; c < KM; ++c) {
                xv[c] = x[c];
                rv[c] = r[c];
                pv[c] = p[c];
                qv[c] = q[c];
            }
#pragma unroll
            for (int c = 0; c < KM; ++c) {
                const double xn = on[c] ? fma(al[c], pv[c], xv[c]) : xv[c];
                const double rn = on[c] ? fma(-al[c], qv[c], rv[c]) : rv[c];
                x[c] = xn;
                r[c] = rn;
                acc[c] = fma(rn, rn, acc[c]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < KM; ++c)
                if (c < k && on[c]) {
                    x[c] = fma(al[c], p[c], x[c]);
                    const double rn = fma(-al[c], q[c], r[c]);
                    r[c] = rn;
                    acc[c] = fma(rn, rn, acc[c]);
                }
        }
    }
    mc_block_partials(acc, part);
}

// beta_c = rho'_c / rho_c, rho_c = rho'_c, the stop tests of the iterating
// columns, and the loop condition: another step while a column iterates
__global__ void __launch_bounds__(kMcFinal)
    mc_beta_kernel(int nblocks, const double* __restrict__ part, MultiState* s, cudaGraphConditionalHandle h)
{
    __shared__ int more;
    if (threadIdx.x == 0) more = 0;
    __syncthreads();
    const int c = threadIdx.x >> 5;
    if (c < s->k) {
        const double rr = mc_column_total(part, nblocks, c);
        if ((threadIdx.x & 31) == 0 && s->phase[c] == kMcIterating) {
            if (!(rr == rr)) {
                s->phase[c] = kMcDone;
                s->status[c] = GKO_ERR_BREAKDOWN;
            } else {
                s->beta[c] = rr / s->rho[c];
                s->rho[c] = rr;
                if (sqrt(rr) <= s->tol * s->stop_ref[c]) {
                    s->phase[c] = kMcConverged;
                } else if (s->iters[c] >= s->maxit) {
                    s->phase[c] = kMcDone;
                    s->status[c] = GKO_ERR_NOT_CONVERGED;
                } else {
                    atomicOr(&more, 1);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && !more) cudaGraphSetConditional(h, 0);
}

// P = R + beta P for the iterating columns (initial: P = R for every
// column); with k == KM a row's loads precede its stores and stopped columns
// are kept by a select
template <int KM>
__global__ void __launch_bounds__(kMcThreads)
    mc_pupdate_kernel(int64_t n, int k, double* __restrict__ P, const double* __restrict__ R, const MultiState* s,
                      int initial)
{
    __shared__ double be_s[kMcMaxK];
    __shared__ int on_s[kMcMaxK];
    if (threadIdx.x < kMcMaxK) {
        const bool it = threadIdx.x < k && (initial || s->phase[threadIdx.x] == kMcIterating);
        on_s[threadIdx.x] = it;
        be_s[threadIdx.x] = initial ? 0.0 : (it ? s->beta[threadIdx.x] : 0.0);
    }
    __syncthreads();
    double be[KM];
    bool on[KM];
#pragma unroll
    for (int c = 0; c < KM; ++c) {
        be[c] = be_s[c];
        on[c] = on_s[c] != 0;
    }
    const bool full = k == KM;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kMcThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kMcThreads) {
        double* p = P + i * k;
        const double* r = R + i * k;
        if (full) {  // every load of the row first, then the stores
            double pv[KM], rv[KM];
#pragma unroll
            for (int c = 0; c < KM; ++c) {
                pv[c] = p[c];
                rv[c] = r[c];
            }
#pragma unroll
            for (int c = 0; c < KM; ++c) p[c] = on[c] ? fma(be[c], pv[c], rv[c]) : pv[c];
        } else {
#pragma unroll
            for (int c = 0; c < KM; ++c)
                if (c < k && on[c]) p[c] = fma(be[c], p[c], r[c]);
        }
    }
}

// R = B - A X's squares per column (R already holds B - A X): partial sums
// of R .* R and of B .* B
template <int KM>
__global__ void __launch_bounds__(kMcThreads)
    mc_norms_kernel(int64_t n, int k, const double* __restrict__ R, const double* __restrict__ B, int64_t ldb,
                    double* __restrict__ part_r, double* __restrict__ part_b)
{
    double acc[KM];
#pragma unroll
    for (int c = 0; c < KM; ++c) acc[c] = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kMcThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kMcThreads) {
        const double* r = R + i * k;
#pragma unroll
        for (int c = 0; c < KM; ++c)
            if (c < k) acc[c] = fma(r[c], r[c], acc[c]);
    }
    mc_block_partials(acc, part_r);
    if (!B) return;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < KM; ++c) acc[c] = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kMcThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kMcThreads) {
        const double* b = B + i * ldb;
#pragma unroll
        for (int c = 0; c < KM; ++c)
            if (c < k) acc[c] = fma(b[c], b[c], acc[c]);
    }
    mc_block_partials(acc, part_b);
}

// column totals of one or two partial arrays into s->val (and out2)
__global__ void __launch_bounds__(kMcFinal)
    mc_totals_kernel(int nblocks, const double* __restrict__ part, const double* __restrict__ part2, MultiState* s,
                     double* __restrict__ out2)
{
    const int c = threadIdx.x >> 5;
    if (c >= s->k) return;
    const double t = mc_column_total(part, nblocks, c);
    const double t2 = part2 ? mc_column_total(part2, nblocks, c) : 0.0;
    if ((threadIdx.x & 31) == 0) {
        s->val[c] = t;
        if (out2) out2[c] = t2;
    }
}

// Q (ld k) = B (ld ldb), row-major blocks
__global__ void mc_copy_kernel(int64_t n, int k, const double* __restrict__ B, int64_t ldb, double* __restrict__ Q)
{
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n * k;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = e / k;
        Q[e] = B[i * ldb + (e - i * k)];
    }
}

// zero column c of X (a column whose right-hand side is zero)
__global__ void mc_zero_column_kernel(int64_t n, double* __restrict__ X, int64_t ldx, int c)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        X[i * ldx + c] = 0.0;
}

// ---------------------------------------------------------------- host

static int mc_read(MultiState* h, const MultiState* d, cudaStream_t st)
{
    GKO_CUDA(cudaMemcpyAsync(h, d, sizeof(MultiState), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    return GKO_OK;
}

static int mc_write(MultiState* d, const MultiState* h, cudaStream_t st)
{
    GKO_CUDA(cudaMemcpyAsync(d, h, sizeof(MultiState), cudaMemcpyHostToDevice, st));
    return GKO_OK;
}

// KM: column capacity of the row kernels' register accumulators (8 or 32);
// 0: k divides 32 and the element kernels run instead
template <int KM>
static int cg_multi_run(const gko_matrix* A, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx,
                        double tol, int maxit, cudaStream_t st, gko_solve_info* infos)
{
    const int64_t n = A->n_rows;
    auto fill = [&](int c, int it, double res, int status) {
        if (!infos) return;
        infos[c].iterations = it;
        infos[c].outer_iterations = 0;
        infos[c].rel_residual = res;
        infos[c].status = status;
        infos[c].aux = 0;
    };
    if (n == 0) {
        for (int c = 0; c < k; ++c) fill(c, 0, 0.0, GKO_OK);
        return GKO_OK;
    }
    const int kk = static_cast<int>(k);
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(kRedBlocks, (n + kMcThreads - 1) / kMcThreads)));
    Workspace ws(st);
    double *R, *P, *Q, *part, *part2, *bn2;
    MultiState* ds;
    GKO_TRY(ws.get(&R, n * k));
    GKO_TRY(ws.get(&P, n * k));
    GKO_TRY(ws.get(&Q, n * k));
    GKO_TRY(ws.get(&part, static_cast<int64_t>(grid) * kMcMaxK));
    GKO_TRY(ws.get(&part2, static_cast<int64_t>(grid) * kMcMaxK));
    GKO_TRY(ws.get(&bn2, kMcMaxK));
    GKO_TRY(ws.get(&ds, 1));
    const int cgrid = static_cast<int>(std::min<int64_t>((n * k + 255) / 256, static_cast<int64_t>(device_sm_count()) * 16));
    MultiState hs = {};
    hs.k = kk;
    hs.maxit = maxit;
    hs.tol = tol;
    GKO_TRY(mc_write(ds, &hs, st));
    // dst = B - A X, |dst_c|^2 into the state's val[c] (and |b_c|^2 into bn2)
    auto residual = [&](double* dst, bool with_b) -> int {
        mc_copy_kernel<<<cgrid, 256, 0, st>>>(n, kk, B, ldb, dst);
        GKO_TRY(spmm_csr(A, k, X, ldx, dst, k, -1.0, 1.0, st));
        mc_norms_kernel<(KM == 0 ? (kMcMaxK) : KM)><<<grid, kMcThreads, 0, st>>>(n, kk, dst, with_b ? B : nullptr, ldb,
                                                                               part, part2);
        mc_totals_kernel<<<1, kMcFinal, 0, st>>>(grid, part, with_b ? part2 : nullptr, ds, with_b ? bn2 : nullptr);
        GKO_CUDA(cudaGetLastError());
        return GKO_OK;
    };
    GKO_TRY(residual(R, true));
    std::vector<double> hb2(kMcMaxK, 0.0);
    GKO_CUDA(cudaMemcpyAsync(hb2.data(), bn2, kMcMaxK * sizeof(double), cudaMemcpyDeviceToHost, st));
    GKO_TRY(mc_read(&hs, ds, st));
    std::vector<double> bnorm(kk), res(kk, -1.0);
    std::vector<int> checks(kk, 0);
    bool any = false;
    for (int c = 0; c < kk; ++c) {
        bnorm[c] = std::sqrt(hb2[c]);
        const double rn = std::sqrt(hs.val[c]);
        hs.stop_ref[c] = bnorm[c];
        hs.rho[c] = hs.val[c];
        hs.iters[c] = 0;
        if (bnorm[c] == 0.0) {  // x_c = 0 at once
            mc_zero_column_kernel<<<cgrid, 256, 0, st>>>(n, X, ldx, c);
            hs.phase[c] = kMcDone;
            hs.status[c] = GKO_OK;
            res[c] = 0.0;
        } else if (!(rn == rn)) {
            hs.phase[c] = kMcDone;
            hs.status[c] = GKO_ERR_BREAKDOWN;
            res[c] = rn / bnorm[c];
        } else if (rn <= tol * bnorm[c]) {  // the true residual already
            hs.phase[c] = kMcDone;
            hs.status[c] = GKO_OK;
            res[c] = rn / bnorm[c];
        } else if (maxit == 0) {
            hs.phase[c] = kMcDone;
            hs.status[c] = GKO_ERR_NOT_CONVERGED;
            res[c] = rn / bnorm[c];
        } else {
            hs.phase[c] = kMcIterating;
            any = true;
        }
    }
    GKO_TRY(mc_write(ds, &hs, st));
    auto pq = [&](cudaStream_t cs) {
        if constexpr (KM == 0)
            mc_pq_elem_kernel<<<grid, kMcThreads, 0, cs>>>(n * k, kk, P, Q, part);
        else
            mc_pq_partial_kernel<KM><<<grid, kMcThreads, 0, cs>>>(n, kk, P, Q, part);
    };
    auto update = [&](cudaStream_t cs) {
        if constexpr (KM == 0)
            mc_update_elem_kernel<<<grid, kMcThreads, 0, cs>>>(n * k, kk, X, ldx, R, P, Q, ds, part);
        else
            mc_update_kernel<KM><<<grid, kMcThreads, 0, cs>>>(n, kk, X, ldx, R, P, Q, ds, part);
    };
    auto pupdate = [&](cudaStream_t cs, int initial) {
        if constexpr (KM == 0)
            mc_pupdate_elem_kernel<<<grid, kMcThreads, 0, cs>>>(n * k, kk, P, R, ds, initial);
        else
            mc_pupdate_kernel<KM><<<grid, kMcThreads, 0, cs>>>(n, kk, P, R, ds, initial);
    };
    pupdate(st, 1);
    GKO_CUDA(cudaGetLastError());
    if (any) {
        GraphHolder gh;
        GKO_TRY(build_while_graph(&gh, [&](cudaGraphConditionalHandle h, cudaStream_t cs) -> int {
            GKO_TRY(spmm_csr(A, k, P, k, Q, k, 1.0, 0.0, cs));
            pq(cs);
            mc_alpha_kernel<<<1, kMcFinal, 0, cs>>>(grid, part, ds);
            update(cs);
            mc_beta_kernel<<<1, kMcFinal, 0, cs>>>(grid, part, ds, h);
            pupdate(cs, 0);
            GKO_CUDA(cudaGetLastError());
            return GKO_OK;
        }));
        while (true) {
            GKO_CUDA(cudaGraphLaunch(gh.exec, st));
            GKO_TRY(mc_read(&hs, ds, st));
            bool pending = false;
            for (int c = 0; c < kk; ++c) pending |= hs.phase[c] == kMcConverged;
            if (!pending) break;
            // confirm the columns whose recursive residual met the tolerance
            // with the FP64 true residual (Q is free between steps)
            GKO_TRY(residual(Q, false));
            MultiState ht;
            GKO_TRY(mc_read(&ht, ds, st));
            bool again = false;
            for (int c = 0; c < kk; ++c) {
                if (hs.phase[c] != kMcConverged) continue;
                res[c] = std::sqrt(ht.val[c]) / bnorm[c];
                ++checks[c];
                if (res[c] <= tol) {
                    hs.phase[c] = kMcDone;
                    hs.status[c] = GKO_OK;
                } else if (checks[c] >= 4 || hs.iters[c] >= maxit) {
                    hs.phase[c] = kMcDone;
                    hs.status[c] = GKO_ERR_NOT_CONVERGED;
                } else {  // not confirmed: finish the step (p = r + beta p) and go on
                    hs.phase[c] = kMcIterating;
                    res[c] = -1.0;
                    again = true;
                }
            }
            GKO_TRY(mc_write(ds, &hs, st));
            if (!again) break;
            pupdate(st, 0);
            GKO_CUDA(cudaGetLastError());
        }
    }
    // residuals not yet formed (stopped at maxit or on a breakdown)
    bool need = false;
    for (int c = 0; c < kk; ++c) need |= res[c] < 0.0;
    if (need) {
        GKO_TRY(residual(Q, false));
        MultiState ht;
        GKO_TRY(mc_read(&ht, ds, st));
        for (int c = 0; c < kk; ++c)
            if (res[c] < 0.0) res[c] = std::sqrt(ht.val[c]) / bnorm[c];
    }
    GKO_CUDA(cudaStreamSynchronize(st));
    int worst = GKO_OK;
    for (int c = 0; c < kk; ++c) {
        fill(c, hs.iters[c], res[c], hs.status[c]);
        if (hs.status[c] != GKO_OK && worst == GKO_OK) worst = hs.status[c];
    }
    if (worst != GKO_OK) set_error("multi-right-hand-side CG: a column did not converge or broke down");
    return worst;
}

int cg_multi_solve(const gko_matrix* A, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx, double tol,
                   int maxit, cudaStream_t st, gko_solve_info* infos)
{
    // KM = 0: k divides 32, the coalesced element kernels
    if (32 % k == 0) return cg_multi_run<0>(A, k, B, ldb, X, ldx, tol, maxit, st, infos);
    if (k <= 8) return cg_multi_run<8>(A, k, B, ldb, X, ldx, tol, maxit, st, infos);
    return cg_multi_run<32>(A, k, B, ldb, X, ldx, tol, maxit, st, infos);
}

}  // namespace gko

using namespace gko;

extern "C" int gko_cg_multi(const gko_matrix* A, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx,
                            double tol, int maxit, void* stream, gko_solve_info* infos)
{
    if (!A) return fail(GKO_ERR_INVALID_ARG, "NULL handle");
    if (A->n_rows != A->n_cols) return fail(GKO_ERR_DIM_MISMATCH, "CG needs a square matrix");
    if (k < 1 || k > kMcMaxK) return fail(GKO_ERR_INVALID_ARG, "k must be in 1..32");
    if (ldb < k || ldx < k) return fail(GKO_ERR_INVALID_ARG, "leading dimensions must be >= k");
    if (!A->has[GKO_FMT_CSR]) return fail(GKO_ERR_FORMAT_UNAVAILABLE, "the product reads the CSR part");
    if (A->n_rows > 0 && (!B || !X)) return fail(GKO_ERR_INVALID_ARG, "NULL block");
    if (!(tol >= 0.0) || maxit < 0) return fail(GKO_ERR_INVALID_ARG, "tol must be >= 0 and maxit >= 0");
    int dev = -1;
    GKO_CUDA(cudaGetDevice(&dev));
    if (dev != A->device) return fail(GKO_ERR_INVALID_ARG, "handle used on another device than it was created on");
    return cg_multi_solve(A, k, B, ldb, X, ldx, tol, maxit, static_cast<cudaStream_t>(stream), infos);
}
