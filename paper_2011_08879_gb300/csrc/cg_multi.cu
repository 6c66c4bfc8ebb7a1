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
// R, P, Q have ld = k.  One step is six launches inside a CUDA-graph WHILE
// loop:
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

// per-column partial sums of P .* Q (rows by thread)
template <int KM>
__global__ void __launch_bounds__(kMcThreads)
    mc_pq_partial_kernel(int64_t n, int k, const double* __restrict__ P, const double* __restrict__ Q,
                         double* __restrict__ part)
{
    double acc[KM];
#pragma unroll
    for (int c = 0; c < KM; ++c) acc[c] = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kMcThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kMcThreads) {
        const double* p = P + i * k;
        const double* q = Q + i * k;
#pragma unroll
        for (int c = 0; c < KM; ++c)
            if (c < k) acc[c] = fma(p[c], q[c], acc[c]);  // k is uniform: a branch, not a predicate
    }
    mc_block_partials(acc, part);
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

// X += alpha P, R -= alpha Q for the iterating columns (alpha of the others
// is not applied); per-column partial sums of R .* R
template <int KM>
__global__ void __launch_bounds__(kMcThreads)
    mc_update_kernel(int64_t n, int k, double* __restrict__ X, int64_t ldx, double* __restrict__ R,
                     const double* __restrict__ P, const double* __restrict__ Q, const MultiState* s,
                     double* __restrict__ part)
{
    __shared__ double al[kMcMaxK];
    __shared__ int on[kMcMaxK];
    if (threadIdx.x < kMcMaxK) {
        const bool it = threadIdx.x < k && s->phase[threadIdx.x] == kMcIterating;
        on[threadIdx.x] = it;
        al[threadIdx.x] = it ? s->alpha[threadIdx.x] : 0.0;
    }
    __syncthreads();
    double acc[KM];
#pragma unroll
    for (int c = 0; c < KM; ++c) acc[c] = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kMcThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kMcThreads) {
        double* x = X + i * ldx;
        double* r = R + i * k;
        const double* p = P + i * k;
        const double* q = Q + i * k;
#pragma unroll
        for (int c = 0; c < KM; ++c)
            if (c < k && on[c]) {
                const double a = al[c];
                x[c] = fma(a, p[c], x[c]);
                const double rc = fma(-a, q[c], r[c]);
                r[c] = rc;
                acc[c] = fma(rc, rc, acc[c]);
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
// column)
template <int KM>
__global__ void __launch_bounds__(kMcThreads)
    mc_pupdate_kernel(int64_t n, int k, double* __restrict__ P, const double* __restrict__ R, const MultiState* s,
                      int initial)
{
    __shared__ double be[kMcMaxK];
    __shared__ int on[kMcMaxK];
    if (threadIdx.x < kMcMaxK) {
        const bool it = threadIdx.x < k && (initial || s->phase[threadIdx.x] == kMcIterating);
        on[threadIdx.x] = it;
        be[threadIdx.x] = initial ? 0.0 : (it ? s->beta[threadIdx.x] : 0.0);
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * static_cast<int64_t>(kMcThreads) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * kMcThreads) {
        double* p = P + i * k;
        const double* r = R + i * k;
#pragma unroll
        for (int c = 0; c < KM; ++c)
            if (c < k && on[c]) p[c] = fma(be[c], p[c], r[c]);
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

// KM: column capacity of the row kernels' register accumulators (8 or 32)
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
        mc_norms_kernel<KM><<<grid, kMcThreads, 0, st>>>(n, kk, dst, with_b ? B : nullptr, ldb, part, part2);
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
    mc_pupdate_kernel<KM><<<grid, kMcThreads, 0, st>>>(n, kk, P, R, ds, 1);
    GKO_CUDA(cudaGetLastError());
    if (any) {
        GraphHolder gh;
        GKO_TRY(build_while_graph(&gh, [&](cudaGraphConditionalHandle h, cudaStream_t cs) -> int {
            GKO_TRY(spmm_csr(A, k, P, k, Q, k, 1.0, 0.0, cs));
            mc_pq_partial_kernel<KM><<<grid, kMcThreads, 0, cs>>>(n, kk, P, Q, part);
            mc_alpha_kernel<<<1, kMcFinal, 0, cs>>>(grid, part, ds);
            mc_update_kernel<KM><<<grid, kMcThreads, 0, cs>>>(n, kk, X, ldx, R, P, Q, ds, part);
            mc_beta_kernel<<<1, kMcFinal, 0, cs>>>(grid, part, ds, h);
            mc_pupdate_kernel<KM><<<grid, kMcThreads, 0, cs>>>(n, kk, P, R, ds, 0);
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
            mc_pupdate_kernel<KM><<<grid, kMcThreads, 0, st>>>(n, kk, P, R, ds, 0);
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
