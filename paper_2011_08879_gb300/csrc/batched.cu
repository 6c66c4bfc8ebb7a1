// Batched CG: many independent small SPD systems solved by one persistent
// kernel.  Each thread block repeatedly takes the next system from a device
// work queue (systems ordered by decreasing size, so the largest start
// first and the tail is short), keeps the system's vectors in shared
// memory, registers or a per-block scratch (the layouts below), streams the
// system's CSR through L1/L2 every step and runs the Hestenes-Stiefel
// recurrence (the Krylov solver of the paper's Sec. 6.2) to its own
// tolerance.  Dots are block-wide reductions in a fixed order; there is no
// inter-block communication except the queue ticket.  The queue reset and
// the kernel are replayed as one CUDA graph.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace gko {

constexpr int kBatchMaxRows = 4096;

template <int BS>
__device__ __forceinline__ double block_dot_sum(double v, double* red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();  // red may still be read by the previous call
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < BS / 32; ++i) t += red[i];  // every thread, same order
    return t;
}


// One row of q = A v for a system (thread per row, local columns).
// (Taking the rows by decreasing length, so that a warp's rows end together,
// was measured slower: 4.96 against 3.62 ms for 4,096 systems, the warps'
// loads of the matrix no longer falling on neighbouring rows.)
__device__ __forceinline__ double sys_row_dot(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                              const double* __restrict__ val, int32_t base, int i, const double* v)
{
    double acc = 0.0;
    const int32_t k1 = rp[i + 1] - base;
    for (int32_t k = rp[i] - base; k < k1; ++k) acc = fma(val[k], v[col[k]], acc);
    return acc;
}

// Sum of part[0 .. BS), called by warp 0 alone: lane l adds part[l],
// part[l + 32], ..., then the warp's tree; the total lands in lane 0.
// FP64 work is charged per warp instruction, whatever the active lanes, so
// one warp adding for the block (BS / 32 + 4 additions) costs the FP64
// pipe 1 / (BS / 32) of every warp reducing its own share and then all
// warps adding the warp totals.
template <int BS>
__device__ __forceinline__ double warp0_sum(const double* part)
{
    double s = part[threadIdx.x];
#pragma unroll
    for (int k = 1; k < BS / 32; ++k) s += part[threadIdx.x + 32 * k];
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;
}

// Block-wide sum of every thread's v, returned to every thread.
template <int BS>
__device__ __forceinline__ double block_sum_bcast(double v, double* part, double* bc)
{
    part[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        const double s = warp0_sum<BS>(part);
        if (threadIdx.x == 0) *bc = s;
    }
    __syncthreads();
    return *bc;
}

enum { kStepGo = 0, kStepBreakdown = 1, kStepCheck = 2 };

// Layouts by the number NS of the system's vectors in shared memory:
//   NS = 4: x, r, p and q = A p all in shared memory (32 bytes per row);
//   NS = 2: p and q in shared memory, x and r in this block's slice of a
//           global scratch;
//   NS = 1: only p, which the product gathers, in shared memory; x, r and
//           q in the scratch.
// Thread t reads and writes only the entries of x, r and q of its own rows
// t, t + BS, ..., so no barrier guards them and scratch entries stay close
// in L1/L2; with 16 or 8 bytes of shared memory per row, 2x or 4x as many
// systems share an SM.  The product and p.q are one pass over the rows.
// Each step's scalars (alpha, beta, the breakdown and stopping tests) are
// derived once, by thread 0 after warp 0 has added the block's partials,
// and read by the other threads from shared memory.
template <int BS, int NS>
__global__ void __launch_bounds__(BS)
    batched_cg_kernel(int64_t count, const int64_t* __restrict__ row_off, const int32_t* __restrict__ row_ptr,
                      const int32_t* __restrict__ col_all, const double* __restrict__ val_all,
                      const int32_t* __restrict__ order, const int32_t* __restrict__ perm, int32_t* queue,
                      const double* __restrict__ b_all, double* __restrict__ x_all, double tol, int maxit,
                      double* __restrict__ res_out, int32_t* __restrict__ it_out, int32_t* __restrict__ st_out,
                      double* scratch, int max_rows)
{
    static_assert(NS == 1 || NS == 2 || NS == 4, "1, 2 or 4 vectors in shared memory");
    extern __shared__ __align__(16) double sm[];
    double* ps = sm;
    double *qv, *xg, *rg;
    if (NS == 4) {
        qv = sm + max_rows;
        xg = sm + 2 * max_rows;
        rg = sm + 3 * max_rows;
    } else {
        xg = scratch + static_cast<size_t>(blockIdx.x) * (4 - NS) * max_rows;
        rg = xg + max_rows;
        qv = NS == 2 ? sm + max_rows : rg + max_rows;
    }
    __shared__ double part[BS];
    __shared__ double s_alpha, s_beta, s_bc;
    __shared__ int s_code, s_next;

    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        const int qi = s_next;
        if (qi >= count) return;
        const int sys = order[qi];
        const int64_t r0 = row_off[sys];
        const int n = static_cast<int>(row_off[sys + 1] - r0);
        const int32_t* rp = row_ptr + r0;
        const int32_t base = rp[0];
        const int32_t* col = col_all + base;
        const double* val = val_all + base;
        const double* b = b_all + r0;
        double* x = x_all + r0;
        const int32_t* pm = perm + r0;  // b and x are indexed in the caller's row order

        double bb = 0.0;
        for (int i = threadIdx.x; i < n; i += BS) {
            const double xi = x[pm[i]];
            xg[i] = xi;
            ps[i] = xi;  // staged for the gathers of A x
            const double bi = b[pm[i]];
            bb = fma(bi, bi, bb);
        }
        const double bnorm = sqrt(block_sum_bcast<BS>(bb, part, &s_bc));  // its barriers also complete ps
        if (bnorm == 0.0) {
            for (int i = threadIdx.x; i < n; i += BS) x[pm[i]] = 0.0;
            if (threadIdx.x == 0) {
                res_out[sys] = 0.0;
                it_out[sys] = 0;
                st_out[sys] = GKO_OK;
            }
            continue;
        }
        // r = b - A x; p = r once every gather of x is done
        double rr = 0.0;
        for (int i = threadIdx.x; i < n; i += BS) {
            const double ri = b[pm[i]] - sys_row_dot(rp, col, val, base, i, ps);
            rg[i] = ri;
            rr = fma(ri, ri, rr);
        }
        double rho = block_sum_bcast<BS>(rr, part, &s_bc);  // after this, kept up to date by thread 0 only
        for (int i = threadIdx.x; i < n; i += BS) ps[i] = rg[i];
        int status = GKO_ERR_NOT_CONVERGED, iter = 0, checks = 0;
        double true_res = -1.0;
        // ||r|| <= tol ||b|| tested as rho <= (tol ||b||)^2: no FP64 square
        // root per step
        const double thr2 = (tol * bnorm) * (tol * bnorm);
        bool stop = rho <= thr2;
        if (stop) status = GKO_OK;
        while (!stop && iter < maxit) {
            __syncthreads();  // p complete before the product
            double pq = 0.0;
            for (int i = threadIdx.x; i < n; i += BS) {
                const double q = sys_row_dot(rp, col, val, base, i, ps);
                qv[i] = q;
                pq = fma(ps[i], q, pq);
            }
            part[threadIdx.x] = pq;
            __syncthreads();
            if (threadIdx.x < 32) {
                const double t = warp0_sum<BS>(part);
                if (threadIdx.x == 0) {
                    const bool bad = !(t > 0.0);
                    s_code = bad ? kStepBreakdown : kStepGo;
                    if (!bad) s_alpha = rho / t;
                }
            }
            __syncthreads();
            ++iter;
            if (s_code == kStepBreakdown) {
                status = GKO_ERR_BREAKDOWN;
                break;
            }
            const double alpha = s_alpha;
            double rn = 0.0;
            for (int i = threadIdx.x; i < n; i += BS) {
                xg[i] = fma(alpha, ps[i], xg[i]);
                const double ri = fma(-alpha, qv[i], rg[i]);
                rg[i] = ri;
                rn = fma(ri, ri, rn);
            }
            part[threadIdx.x] = rn;
            __syncthreads();  // also: every gather of p done
            if (threadIdx.x < 32) {
                const double u = warp0_sum<BS>(part);
                if (threadIdx.x == 0) {
                    if (!(u == u)) {
                        s_code = kStepBreakdown;
                    } else {
                        s_code = u <= thr2 ? kStepCheck : kStepGo;
                        s_beta = u / rho;
                        rho = u;
                    }
                }
            }
            __syncthreads();
            const int code = s_code;
            if (code == kStepBreakdown) {
                status = GKO_ERR_BREAKDOWN;
                break;
            }
            if (code == kStepCheck) {
                // confirm with the true residual: p parked in q's rows, x staged in ps
                for (int i = threadIdx.x; i < n; i += BS) {
                    qv[i] = ps[i];
                    ps[i] = xg[i];
                }
                __syncthreads();
                double tt = 0.0;
                for (int i = threadIdx.x; i < n; i += BS) {
                    const double ti = b[pm[i]] - sys_row_dot(rp, col, val, base, i, ps);
                    tt = fma(ti, ti, tt);
                }
                true_res = sqrt(block_sum_bcast<BS>(tt, part, &s_bc)) / bnorm;  // every gather of x done
                for (int i = threadIdx.x; i < n; i += BS) ps[i] = qv[i];
                ++checks;
                if (true_res <= tol) {
                    status = GKO_OK;
                    break;
                }
                if (checks >= 4) break;
                true_res = -1.0;
            }
            const double beta = s_beta;
            for (int i = threadIdx.x; i < n; i += BS) ps[i] = fma(beta, ps[i], rg[i]);
        }
        if (true_res < 0.0) {
            __syncthreads();  // no thread still gathers p
            for (int i = threadIdx.x; i < n; i += BS) ps[i] = xg[i];
            __syncthreads();
            double tt = 0.0;
            for (int i = threadIdx.x; i < n; i += BS) {
                const double ti = b[pm[i]] - sys_row_dot(rp, col, val, base, i, ps);
                tt = fma(ti, ti, tt);
            }
            true_res = sqrt(block_sum_bcast<BS>(tt, part, &s_bc)) / bnorm;
        }
        for (int i = threadIdx.x; i < n; i += BS) x[pm[i]] = xg[i];
        if (threadIdx.x == 0) {
            res_out[sys] = true_res;
            it_out[sys] = iter;
            st_out[sys] = status;
        }
    }
}

// Launch of the layouts above.  NS < 4 needs a scratch of (4 - NS) vectors
// of max_rows doubles per resident block: prepare = true only sizes it
// (before a graph capture, where no allocation may run); prepare = false
// launches.
template <int BS, int NS>
static int launch_batched(gko_batch* B, const double* b, double* x, double tol, int maxit, cudaStream_t st,
                          bool prepare)
{
    const size_t smem = NS * static_cast<size_t>(B->max_rows) * sizeof(double);
    GKO_CUDA(smem_limit_once(reinterpret_cast<const void*>(batched_cg_kernel<BS, NS>), static_cast<int>(smem)));
    int per_sm = 0;
    const int sms = device_sm_count();
    GKO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_cg_kernel<BS, NS>, BS, smem));
    if (per_sm < 1) return fail(GKO_ERR_INVALID_ARG, "batched CG: block does not fit on an SM");
    const int64_t grid = std::max<int64_t>(std::min<int64_t>(static_cast<int64_t>(per_sm) * sms, B->count), 1);
    const int64_t need = NS == 4 ? 0 : grid * (4 - NS) * static_cast<int64_t>(B->max_rows);
    if (prepare) {
        if (B->scratch_len >= need) return GKO_OK;
        dev_free(B->scratch);  // synchronises: no earlier solve still uses it
        B->scratch = nullptr;
        B->scratch_len = 0;
        GKO_TRY(dev_alloc(&B->scratch, need));
        B->scratch_len = need;
        return GKO_OK;
    }
    if (B->scratch_len < need) return fail(GKO_ERR_INVALID_ARG, "batched CG: scratch not prepared");
    GKO_CUDA(cudaMemsetAsync(B->queue, 0, sizeof(int32_t), st));
    batched_cg_kernel<BS, NS><<<static_cast<unsigned>(grid), BS, smem, st>>>(
        B->count, B->row_off, B->row_ptr, B->col, B->val, B->order, B->perm, B->queue, b, x, tol, maxit, B->res, B->iters,
        B->status, B->scratch, B->max_rows);
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}

// ---------------------------------------------------------------------------
// Register-resident variant: thread t owns rows t, t + BS, ..., t + (R-1) BS
// of its system (R rows per thread, BS * R >= the largest system), keeps x,
// r and (A p) of those rows in registers and only the direction p, which
// the product gathers, in shared memory (8 bytes per row instead of 32), so
// more blocks share an SM.  Same recurrence, stops and outputs as
// batched_cg_kernel; the autotuner times every layout.

template <int BS, int R>
__device__ __forceinline__ void sys_spmv_reg(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                             const double* __restrict__ val, int32_t base, const double* v, double* q)
{
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int i = threadIdx.x + k * BS;
        double acc = 0.0;
        if (i < n) {
            const int32_t k1 = rp[i + 1] - base;
            for (int32_t kk = rp[i] - base; kk < k1; ++kk) acc = fma(val[kk], v[col[kk]], acc);
        }
        q[k] = acc;
    }
}

// sum over the thread's rows of (b_i - (A v)_i)^2
template <int BS, int R>
__device__ __forceinline__ double sys_resid2_reg(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                 const double* __restrict__ val, int32_t base, const double* v,
                                                 const double* __restrict__ b, const int32_t* __restrict__ pm)
{
    double tt = 0.0;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int i = threadIdx.x + k * BS;
        if (i < n) {
            double acc = 0.0;
            const int32_t k1 = rp[i + 1] - base;
            for (int32_t kk = rp[i] - base; kk < k1; ++kk) acc = fma(val[kk], v[col[kk]], acc);
            const double t = b[pm[i]] - acc;
            tt = fma(t, t, tt);
        }
    }
    return tt;
}

template <int BS, int R>
__global__ void __launch_bounds__(BS)
    batched_cg_reg_kernel(int64_t count, const int64_t* __restrict__ row_off, const int32_t* __restrict__ row_ptr,
                          const int32_t* __restrict__ col_all, const double* __restrict__ val_all,
                          const int32_t* __restrict__ order, const int32_t* __restrict__ perm, int32_t* queue,
                          const double* __restrict__ b_all, double* __restrict__ x_all, double tol, int maxit,
                          double* __restrict__ res_out, int32_t* __restrict__ it_out, int32_t* __restrict__ st_out)
{
    extern __shared__ __align__(16) double ps[];  // the direction p (or x while a residual is formed)
    __shared__ double red[BS / 32];
    __shared__ int s_next;

    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        const int qi = s_next;
        if (qi >= count) return;
        const int sys = order[qi];
        const int64_t r0 = row_off[sys];
        const int n = static_cast<int>(row_off[sys + 1] - r0);
        const int32_t* rp = row_ptr + r0;
        const int32_t base = rp[0];
        const int32_t* col = col_all + base;
        const double* val = val_all + base;
        const double* b = b_all + r0;
        double* x = x_all + r0;
        const int32_t* pm = perm + r0;  // b and x are indexed in the caller's row order

        double xr[R], rr[R], qr[R];
        double bb = 0.0;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int i = threadIdx.x + k * BS;
            xr[k] = i < n ? x[pm[i]] : 0.0;
            rr[k] = i < n ? b[pm[i]] : 0.0;
            bb = fma(rr[k], rr[k], bb);
        }
        const double bnorm = sqrt(block_dot_sum<BS>(bb, red));
        if (bnorm == 0.0) {
#pragma unroll
            for (int k = 0; k < R; ++k)
                if (threadIdx.x + k * BS < n) x[pm[threadIdx.x + k * BS]] = 0.0;
            if (threadIdx.x == 0) {
                res_out[sys] = 0.0;
                it_out[sys] = 0;
                st_out[sys] = GKO_OK;
            }
            continue;
        }
        // r = b - A x (the product gathers x, staged in ps); then p = r
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (threadIdx.x + k * BS < n) ps[threadIdx.x + k * BS] = xr[k];
        __syncthreads();
        sys_spmv_reg<BS, R>(n, rp, col, val, base, ps, qr);
        __syncthreads();  // every gather of x done before ps becomes p
        double rho = 0.0;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int i = threadIdx.x + k * BS;
            if (i < n) {
                rr[k] -= qr[k];
                ps[i] = rr[k];
                rho = fma(rr[k], rr[k], rho);
            }
        }
        rho = block_dot_sum<BS>(rho, red);  // its barrier also completes p
        int status = GKO_ERR_NOT_CONVERGED, iter = 0, checks = 0;
        double true_res = -1.0;
        // ||r|| <= tol ||b|| tested as rho <= (tol ||b||)^2: no FP64 square
        // root per step (FP64 work is charged per warp instruction)
        const double thr2 = (tol * bnorm) * (tol * bnorm);
        bool stop = rho <= thr2;
        if (stop) status = GKO_OK;
        while (!stop && iter < maxit) {
            sys_spmv_reg<BS, R>(n, rp, col, val, base, ps, qr);
            double pq = 0.0;
#pragma unroll
            for (int k = 0; k < R; ++k)
                if (threadIdx.x + k * BS < n) pq = fma(ps[threadIdx.x + k * BS], qr[k], pq);
            pq = block_dot_sum<BS>(pq, red);
            ++iter;
            if (!(pq > 0.0)) {
                status = GKO_ERR_BREAKDOWN;
                break;
            }
            const double alpha = rho / pq;
            double rn = 0.0;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const int i = threadIdx.x + k * BS;
                if (i < n) {
                    xr[k] = fma(alpha, ps[i], xr[k]);
                    rr[k] = fma(-alpha, qr[k], rr[k]);
                    rn = fma(rr[k], rr[k], rn);
                }
            }
            const double rho_new = block_dot_sum<BS>(rn, red);  // every read of p done past its barrier
            if (!(rho_new == rho_new)) {
                status = GKO_ERR_BREAKDOWN;
                break;
            }
            if (rho_new <= thr2) {
                // confirm with the true residual: stage x in ps, keeping p's own rows in qr
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const int i = threadIdx.x + k * BS;
                    if (i < n) {
                        qr[k] = ps[i];
                        ps[i] = xr[k];
                    }
                }
                __syncthreads();
                const double tt = sys_resid2_reg<BS, R>(n, rp, col, val, base, ps, b, pm);
                true_res = sqrt(block_dot_sum<BS>(tt, red)) / bnorm;  // every gather of x done past its barrier
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (threadIdx.x + k * BS < n) ps[threadIdx.x + k * BS] = qr[k];
                ++checks;
                if (true_res <= tol) {
                    status = GKO_OK;
                    break;
                }
                if (checks >= 4) break;
                true_res = -1.0;
            }
            const double beta = rho_new / rho;
            rho = rho_new;
#pragma unroll
            for (int k = 0; k < R; ++k)
                if (threadIdx.x + k * BS < n) ps[threadIdx.x + k * BS] = fma(beta, ps[threadIdx.x + k * BS], rr[k]);
            __syncthreads();  // p complete before the next product
        }
        if (true_res < 0.0) {
            __syncthreads();  // no thread still gathers p
#pragma unroll
            for (int k = 0; k < R; ++k)
                if (threadIdx.x + k * BS < n) ps[threadIdx.x + k * BS] = xr[k];
            __syncthreads();
            const double tt = sys_resid2_reg<BS, R>(n, rp, col, val, base, ps, b, pm);
            true_res = sqrt(block_dot_sum<BS>(tt, red)) / bnorm;
        }
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (threadIdx.x + k * BS < n) x[pm[threadIdx.x + k * BS]] = xr[k];
        if (threadIdx.x == 0) {
            res_out[sys] = true_res;
            it_out[sys] = iter;
            st_out[sys] = status;
        }
    }
}

template <int BS, int R>
static int launch_batched_reg(gko_batch* B, const double* b, double* x, double tol, int maxit, cudaStream_t st)
{
    if (B->max_rows > BS * R) return fail(GKO_ERR_INVALID_ARG, "batched CG: systems larger than block x rows");
    const size_t smem = static_cast<size_t>(B->max_rows) * sizeof(double);
    GKO_CUDA(smem_limit_once(reinterpret_cast<const void*>(batched_cg_reg_kernel<BS, R>), static_cast<int>(smem)));
    int per_sm = 0;
    const int sms = device_sm_count();
    GKO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_cg_reg_kernel<BS, R>, BS, smem));
    if (per_sm < 1) return fail(GKO_ERR_INVALID_ARG, "batched CG: block does not fit on an SM");
    const int64_t grid = std::min<int64_t>(static_cast<int64_t>(per_sm) * sms, B->count);
    GKO_CUDA(cudaMemsetAsync(B->queue, 0, sizeof(int32_t), st));
    batched_cg_reg_kernel<BS, R><<<static_cast<unsigned>(std::max<int64_t>(grid, 1)), BS, smem, st>>>(
        B->count, B->row_off, B->row_ptr, B->col, B->val, B->order, B->perm, B->queue, b, x, tol, maxit, B->res, B->iters,
        B->status);
    GKO_CUDA(cudaGetLastError());
    return GKO_OK;
}


// Launch configurations: block sizes 64..1024 with the vectors in shared
// memory; -BS for the register-resident layout of BS threads with R =
// 1024 / BS rows per thread.
static int launch_any(gko_batch* B, int bs, const double* b, double* x, double tol, int maxit, cudaStream_t st,
                      bool prepare = false)
{
    constexpr int P = GKO_BATCH_SHARED_P, PQ = GKO_BATCH_SHARED_PQ;
    switch (bs) {
        case P | 32: return launch_batched<32, 1>(B, b, x, tol, maxit, st, prepare);
        case P | 64: return launch_batched<64, 1>(B, b, x, tol, maxit, st, prepare);
        case P | 128: return launch_batched<128, 1>(B, b, x, tol, maxit, st, prepare);
        case P | 256: return launch_batched<256, 1>(B, b, x, tol, maxit, st, prepare);
        case PQ | 32: return launch_batched<32, 2>(B, b, x, tol, maxit, st, prepare);
        case PQ | 64: return launch_batched<64, 2>(B, b, x, tol, maxit, st, prepare);
        case PQ | 128: return launch_batched<128, 2>(B, b, x, tol, maxit, st, prepare);
        case PQ | 256: return launch_batched<256, 2>(B, b, x, tol, maxit, st, prepare);
        case 64: return launch_batched<64, 4>(B, b, x, tol, maxit, st, prepare);
        case 128: return launch_batched<128, 4>(B, b, x, tol, maxit, st, prepare);
        case 256: return launch_batched<256, 4>(B, b, x, tol, maxit, st, prepare);
        case 512: return launch_batched<512, 4>(B, b, x, tol, maxit, st, prepare);
        case 1024: return launch_batched<1024, 4>(B, b, x, tol, maxit, st, prepare);
    }
    if (prepare) return GKO_OK;  // the register layout needs no scratch
    switch (bs) {
        case -128: return launch_batched_reg<128, 8>(B, b, x, tol, maxit, st);
        case -256: return launch_batched_reg<256, 4>(B, b, x, tol, maxit, st);
        case -512: return launch_batched_reg<512, 2>(B, b, x, tol, maxit, st);
        case -1024: return launch_batched_reg<1024, 1>(B, b, x, tol, maxit, st);
    }
    return fail(GKO_ERR_INVALID_ARG,
                "block_size must be 0, 64..1024, -128..-1024, or GKO_BATCH_SHARED_P / _PQ | 32..256");
}

// run [queue reset + kernel] as a captured CUDA graph; the instantiated
// graph is kept in the batch and relaunched while block size, vectors,
// tolerance and iteration limit are those it was captured with
static int run_graph(gko_batch* B, int bs, const double* b, double* x, double tol, int maxit, cudaStream_t st)
{
    if (B->graph && B->graph_bs == bs && B->graph_b == b && B->graph_x == x && B->graph_tol == tol &&
        B->graph_maxit == maxit) {
        GKO_CUDA(cudaGraphLaunch(B->graph, st));
        return GKO_OK;
    }
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    GKO_TRY(launch_any(B, bs, b, x, tol, maxit, st, true));
    cudaStream_t cap;
    GKO_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    int s = GKO_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        s = launch_any(B, bs, b, x, tol, maxit, cap);
        e = cudaStreamEndCapture(cap, &g);
    }
    if (e == cudaSuccess && s == GKO_OK) e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess && s == GKO_OK) e = cudaGraphLaunch(ge, st);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (s != GKO_OK || e != cudaSuccess) {
        if (ge) cudaGraphExecDestroy(ge);
        if (s != GKO_OK) return s;
        return cuda_fail(e, "batched CG graph");
    }
    B->graph = ge;
    B->graph_bs = bs;
    B->graph_b = b;
    B->graph_x = x;
    B->graph_tol = tol;
    B->graph_maxit = maxit;
    return GKO_OK;
}

}  // namespace gko

using namespace gko;

extern "C" {

int gko_batch_create(int64_t count, const int64_t* row_off, const int32_t* row_ptr, const int32_t* col,
                     const double* val, int on_device, void* stream, gko_batch** out)
{
    if (!out || !row_off || !row_ptr) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (count < 1 || count > INT32_MAX) return fail(GKO_ERR_INVALID_ARG, "count must be in [1, 2^31)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    std::vector<int64_t> ro(count + 1);
    GKO_CUDA(cudaMemcpy(ro.data(), row_off, (count + 1) * sizeof(int64_t), kind));
    if (ro[0] != 0) return fail(GKO_ERR_INVALID_ARG, "row_off[0] must be 0");
    int max_rows = 0;
    for (int64_t s = 0; s < count; ++s) {
        const int64_t n = ro[s + 1] - ro[s];
        if (n < 1 || n > kBatchMaxRows) return fail(GKO_ERR_INVALID_ARG, "systems must have 1..4096 rows");
        max_rows = std::max<int>(max_rows, static_cast<int>(n));
    }
    const int64_t n_rows = ro[count];
    if (n_rows >= INT32_MAX) return fail(GKO_ERR_INVALID_ARG, "too many rows");
    int32_t last = 0;
    GKO_CUDA(cudaMemcpy(&last, row_ptr + n_rows, sizeof(int32_t), kind));
    const int64_t nnz = last;
    if (nnz > 0 && (!col || !val)) return fail(GKO_ERR_INVALID_ARG, "NULL array");
    // host copies of the systems, validated, then renumbered
    std::vector<int32_t> hrp(n_rows + 1), hcol(nnz), hperm(n_rows);
    std::vector<double> hval(nnz);
    GKO_CUDA(cudaMemcpy(hrp.data(), row_ptr, (n_rows + 1) * sizeof(int32_t), kind));
    if (nnz) {
        GKO_CUDA(cudaMemcpy(hcol.data(), col, nnz * sizeof(int32_t), kind));
        GKO_CUDA(cudaMemcpy(hval.data(), val, nnz * sizeof(double), kind));
    }
    if (hrp[0] != 0) return fail(GKO_ERR_INVALID_MATRIX, "row_ptr[0] must be 0");
    for (int64_t i = 0; i < n_rows; ++i)
        if (hrp[i + 1] < hrp[i]) return fail(GKO_ERR_INVALID_MATRIX, "row_ptr must be non-decreasing");
    for (int64_t sy = 0; sy < count; ++sy) {
        const int64_t ns = ro[sy + 1] - ro[sy];
        for (int64_t k = hrp[ro[sy]]; k < hrp[ro[sy + 1]]; ++k)
            if (hcol[k] < 0 || hcol[k] >= ns) return fail(GKO_ERR_INVALID_MATRIX, "column index outside its system");
    }
    // Every system is stored renumbered, P A P^T with its rows in order of
    // decreasing length (stable): the kernels give a thread one row at a time
    // and a warp's FMA loop runs to its longest row, so rows of like length
    // side by side waste fewer FP64 slots (on the 4,096-system benchmark
    // batch: 1.06 instead of 1.53 issued per stored entry).  perm[r0 + k] is
    // the caller's row of stored row k; the kernels gather b and x and
    // scatter x through it.
    std::vector<int32_t> nrp(n_rows + 1), ncol(nnz), inv;
    std::vector<double> nval(nnz);
    nrp[0] = 0;
    for (int64_t sy = 0; sy < count; ++sy) {
        const int64_t r0 = ro[sy], ns = ro[sy + 1] - r0;
        int32_t* pm = hperm.data() + r0;
        std::iota(pm, pm + ns, 0);
        std::stable_sort(pm, pm + ns, [&](int32_t a, int32_t c) {
            return hrp[r0 + a + 1] - hrp[r0 + a] > hrp[r0 + c + 1] - hrp[r0 + c];
        });
        inv.assign(ns, 0);
        for (int64_t k = 0; k < ns; ++k) inv[pm[k]] = static_cast<int32_t>(k);
        std::vector<std::pair<int32_t, double>> rowbuf;
        for (int64_t k = 0; k < ns; ++k) {
            const int64_t src = r0 + pm[k];
            rowbuf.clear();
            for (int64_t e = hrp[src]; e < hrp[src + 1]; ++e) rowbuf.emplace_back(inv[hcol[e]], hval[e]);
            std::stable_sort(rowbuf.begin(), rowbuf.end(),
                             [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& c) {
                                 return a.first < c.first;
                             });
            int64_t d = nrp[r0 + k];
            for (const auto& pr : rowbuf) {
                ncol[d] = pr.first;
                nval[d] = pr.second;
                ++d;
            }
            nrp[r0 + k + 1] = static_cast<int32_t>(d);
        }
    }
    gko_batch* B = new gko_batch();
    auto cleanup = [&](int s) {
        gko_batch_destroy(B);
        return s;
    };
    B->count = count;
    B->n_rows = n_rows;
    B->nnz = nnz;
    B->max_rows = max_rows;
    GKO_CUDA(cudaGetDevice(&B->device));
    int s;
    if ((s = dev_alloc(&B->row_off, count + 1)) || (s = dev_alloc(&B->row_ptr, n_rows + 1)) ||
        (s = dev_alloc(&B->col, nnz)) || (s = dev_alloc(&B->val, nnz)) || (s = dev_alloc(&B->order, count)) ||
        (s = dev_alloc(&B->queue, 1)) || (s = dev_alloc(&B->res, count)) || (s = dev_alloc(&B->iters, count)) ||
        (s = dev_alloc(&B->status, count)) || (s = dev_alloc(&B->d_err, 1)) || (s = dev_alloc(&B->perm, n_rows)))
        return cleanup(s);
    // work-queue order: decreasing size, ties by index
    std::vector<int32_t> ord(count);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int32_t a, int32_t c) { return ro[a + 1] - ro[a] > ro[c + 1] - ro[c]; });
    cudaError_t e = cudaMemcpyAsync(B->row_off, ro.data(), (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->row_ptr, nrp.data(), (n_rows + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(B->col, ncol.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(B->val, nval.data(), nnz * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->perm, hperm.data(), n_rows * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B->order, ord.data(), count * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "copying the batch"));
    *out = B;
    return GKO_OK;
}

int gko_batch_destroy(gko_batch* B)
{
    if (!B) return GKO_OK;
    dev_free(B->row_off);
    dev_free(B->row_ptr);
    dev_free(B->col);
    dev_free(B->val);
    dev_free(B->order);
    dev_free(B->queue);
    dev_free(B->res);
    dev_free(B->iters);
    dev_free(B->status);
    dev_free(B->d_err);
    dev_free(B->perm);
    dev_free(B->scratch);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    delete B;
    return GKO_OK;
}

int gko_cg_batched(gko_batch* B, const double* b, double* x, double tol, int maxit, int block_size, void* stream,
                   gko_solve_info* infos)
{
    if (!B || !b || !x) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    if (!(tol >= 0.0) || maxit < 0) return fail(GKO_ERR_INVALID_ARG, "tol must be >= 0 and maxit >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // untuned: p alone in shared memory at 128 threads, the layout with the
    // most resident systems per SM (fastest on the 4,096-system benchmark)
    int bs = block_size ? block_size : (B->best_block ? B->best_block : GKO_BATCH_SHARED_P | 128);
    GKO_TRY(run_graph(B, bs, b, x, tol, maxit, st));
    std::vector<double> res(B->count);
    std::vector<int32_t> it(B->count), stv(B->count);
    GKO_CUDA(cudaMemcpyAsync(res.data(), B->res, B->count * sizeof(double), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaMemcpyAsync(it.data(), B->iters, B->count * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaMemcpyAsync(stv.data(), B->status, B->count * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    int worst = GKO_OK;
    for (int64_t s = 0; s < B->count; ++s) {
        if (stv[s] != GKO_OK && (worst == GKO_OK || stv[s] == GKO_ERR_BREAKDOWN)) worst = stv[s];
        if (infos) {
            infos[s].iterations = it[s];
            infos[s].outer_iterations = 0;
            infos[s].rel_residual = res[s];
            infos[s].status = stv[s];
            infos[s].aux = 0;
        }
    }
    if (worst != GKO_OK) set_error("batched CG: some systems did not converge");
    return worst;
}

int gko_batch_autotune(gko_batch* B, const double* b, double* x, double tol, int maxit, void* stream, int* best)
{
    if (!B || !b || !x || !best) return fail(GKO_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* x0 = nullptr;
    GKO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&x0), B->n_rows * sizeof(double), st));
    GKO_CUDA(cudaMemcpyAsync(x0, x, B->n_rows * sizeof(double), cudaMemcpyDeviceToDevice, st));
    cudaEvent_t e0, e1;
    GKO_CUDA(cudaEventCreate(&e0));
    GKO_CUDA(cudaEventCreate(&e1));
    float best_ms = 0.0f;
    int best_bs = 0;
    constexpr int P = GKO_BATCH_SHARED_P, PQ = GKO_BATCH_SHARED_PQ;
    const int cands[] = {64,      128,      256,      512,     1024,     -128,     -256,    -512,
                         -1024,   P | 32,   P | 64,   P | 128, P | 256,  PQ | 32,  PQ | 64, PQ | 128,
                         PQ | 256};
    for (int bs : cands) {
        if (bs < 0 && B->max_rows > 1024) continue;  // R = 1024 / BS rows per thread must cover the systems
        float tot = 0.0f;
        int s = GKO_OK;
        for (int rep = 0; rep < 3 && s == GKO_OK; ++rep) {
            GKO_CUDA(cudaMemcpyAsync(x, x0, B->n_rows * sizeof(double), cudaMemcpyDeviceToDevice, st));
            GKO_CUDA(cudaEventRecord(e0, st));
            s = run_graph(B, bs, b, x, tol, maxit, st);
            GKO_CUDA(cudaEventRecord(e1, st));
            GKO_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            GKO_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) tot += ms;  // first run warms up
        }
        if (s != GKO_OK) continue;
        if (best_bs == 0 || tot < best_ms) {
            best_ms = tot;
            best_bs = bs;
        }
    }
    GKO_CUDA(cudaMemcpyAsync(x, x0, B->n_rows * sizeof(double), cudaMemcpyDeviceToDevice, st));
    GKO_CUDA(cudaFreeAsync(x0, st));
    GKO_CUDA(cudaStreamSynchronize(st));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!best_bs) return fail(GKO_ERR_INVALID_ARG, "no block size could be launched");
    B->best_block = best_bs;  // negative: the register-resident layout
    *best = best_bs;
    return GKO_OK;
}

}  // extern "C"
